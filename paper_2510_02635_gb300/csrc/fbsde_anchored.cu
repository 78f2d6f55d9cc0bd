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
//
// Kernels: the contractions of FP32 solves with M >= 1024 run on the tensor cores
// (k_gemm_tc, split TF32, fbsde_tcgemm.cuh), the CG pass's P V^T with the column pass fused
// into its epilogue; smaller or FP64 solves use the SIMT k_gemm and k_anc_columns.  The
// per-anchor d-vector kernels run one warp (setup, Newton) or one block (the CG pass of rows up
// to 1024 chunks, its vectors in registers) per anchor.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <list>
#include <mutex>
#include <vector>

#include "fbsde_kernels.cuh"
#include "fbsde_tcgemm.cuh"

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
// Band (batch reading, see dev::Band): NT products skip tiles with no used entry; TN
// products write a zero partial for a split whose rows miss the band of the tile's anchors.
template <typename Real, bool TN>
__global__ void __launch_bounds__(256) k_gemm(int Mr, int Nc, int K, int kc,
                                              const Real *__restrict__ A, int lda,
                                              const Real *__restrict__ B, int ldb,
                                              Real *__restrict__ C, int ldc, dev::Band band)
{
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ Real As[BK][BM + 1];
    __shared__ Real Bs[BK][BN + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int r0 = blockIdx.y * BM, c0 = blockIdx.x * BN;
    int kb = blockIdx.z * kc, ke = min(K, kb + kc);
    if (!TN && !band.hits(r0, min(Mr, r0 + BM), c0, min(Nc, c0 + BN))) return;
    if (TN && !band.hits(kb, ke, r0, min(Mr, r0 + BM))) ke = kb;   // zero partial
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
//           With a batch of Kb < M particles per anchor (random-batch reading of Remark
//           2.1), w_jm = 0 outside the cyclic window j = (m + q) mod M, q < Kb.
//   mode 1: T_jm = w_jm (G_jm - A_m . v_m) / W_m stored in T; sum T.
constexpr int kRowChunk = 64;
template <typename Real>
__global__ void k_anc_columns(Params p, int mode, double rho_ref, long long Kb,
                              const Real *__restrict__ G, const double *__restrict__ pn,
                              const double *__restrict__ an, const double *__restrict__ Y,
                              Real *__restrict__ W, Real *__restrict__ T, const Anchor *st,
                              double *part)
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
#pragma unroll 8
        for (long long j = j0; j < j1; ++j) {
            long long off = j - m;   // position of particle j in anchor m's window
            if (off < 0) off += p.M;
            Real w = Real(0);
            if (off < Kb) {   // outside the window the product entry may not be computed
                const Real rho = max((Real)pn[j] + am - Real(2) * G[(size_t)j * p.M + m], Real(0));
                w = exp((rho - ref) * scale);
                sw += w;
                swy += w * (Real)Y[j];
                swr += w * rho;
            }
            W[(size_t)j * p.M + m] = w;
        }
        o[0] = (double)sw;
        o[1] = (double)swy;
        o[2] = (double)swr;
    } else {
        const Anchor &a = st[m];
        if (a.done) return;
        const Real inv = (Real)(1.0 / a.W), ap = (Real)a.ap;
        Real sum = 0;
#pragma unroll 8
        for (long long j = j0; j < j1; ++j) {
            const size_t ix = (size_t)j * p.M + m;
            long long off = j - m;
            if (off < 0) off += p.M;
            const Real t = off < Kb ? W[ix] * (G[ix] - ap) * inv : Real(0);
            T[ix] = t;
            sum += t;
        }
        o[0] = (double)sum;
    }
}

// Sum over the nsplit partial products X[z * split + ix], z in order, in the stream
// precision (eight loads in flight): the partials are stream-precision sums themselves, and
// on this part the FP64 pipe is a small fraction of the FP32 one.
template <typename Real>
__device__ __forceinline__ Real split_sum(const Real *X, size_t split, size_t ix, int nsplit)
{
    Real g = Real(0);
    int z = 0;
    for (; z + 8 <= nsplit; z += 8) {
        Real t[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) t[u] = X[(z + u) * split + ix];
#pragma unroll
        for (int u = 0; u < 8; ++u) g += t[u];
    }
    for (; z < nsplit; ++z) g += X[z * split + ix];
    return g;
}

// The per-anchor d-vector kernels run one warp per anchor, kAncWarps anchors per block, with
// warp-only tree sums: on this part the FP64 pipe is a small fraction of the FP32 one, and
// block-wide FP64 reductions repeated by every thread cost more than the element work.
constexpr int kAncWarps = 8;
template <typename T, int NV> __device__ __forceinline__ void warp_sums(T (&v)[NV])
{
#pragma unroll
    for (int i = 0; i < NV; ++i)
#pragma unroll
        for (int o = 16; o; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
}

// Per anchor: S, rhs, lambda, and the CG start x = 0, r = p = rhs.  The per-anchor
// d-vectors (S, rhs, x, r, p, q) and their element arithmetic are in the stream precision:
// on the FP32 path the CG passes then run on the FP32 pipe at half the bytes (the FP64 pipe
// is a small fraction of it on this part); the scalars of each anchor stay FP64.
template <typename Real>
__global__ void __launch_bounds__(32 * kAncWarps) k_anc_setup(Params p, int nrc, int nsplit,
                                                              const Real *A, const Real *G2,
                                                              const Real *G3, const double *part,
                                                              Anchor *st, Real *S, Real *rhs,
                                                              Real *x, Real *r, Real *pv)
{
    const int lane = threadIdx.x & 31;
    const int m = blockIdx.x * kAncWarps + (threadIdx.x >> 5);
    if (m >= p.M) return;
    Anchor &a = st[m];
    double w[3] = {0.0, 0.0, 0.0};   // column sums of the weights: lane-strided chunks in
                                     // order, then the warp tree
    for (int c = lane; c < nrc; c += 32) {
        const double *o = part + ((size_t)c * p.M + m) * 3;
        w[0] += o[0];
        w[1] += o[1];
        w[2] += o[2];
    }
    warp_sums(w);
    const double invW = 1.0 / w[0], cm = w[1] / w[0];
    const Real invWr = (Real)invW, cmr = (Real)cm;
    const size_t o = (size_t)m * p.ld, split = (size_t)p.M * p.ld;
    Real acc[4] = {Real(0), Real(0), Real(0), Real(0)};   // |S|^2, |rhs|^2, S . rhs, A . rhs
    for (int i = lane; i < p.ld; i += 32) {
        const Real g2 = split_sum(G2, split, o + i, nsplit) * invWr;
        const Real g3 = split_sum(G3, split, o + i, nsplit);
        const Real ai = A[o + i];
        const Real sv = g2 - ai;
        const Real b = g3 * invWr - cmr * g2;
        S[o + i] = sv;
        rhs[o + i] = b;
        x[o + i] = Real(0);
        r[o + i] = b;
        pv[o + i] = b;
        acc[0] += sv * sv;
        acc[1] += b * b;
        acc[2] += sv * b;
        acc[3] += ai * b;
    }
    warp_sums(acc);
    if (lane == 0) {
        a.W = w[0];
        a.c = cm;
        a.lam = p.ridge_rel * (w[2] * invW - acc[0]) / p.d;
        a.rr = acc[1];
        a.rhs2 = acc[1];
        a.sp = acc[2];
        a.ap = acc[3];
        a.iters = 0;
        a.status = 0;
        a.done = acc[1] == 0.0 ? 1 : 0;
    }
}

// One CG pass per anchor:
// q = G_m - colsum_m A_m - S_m (S_m . p_m) + lambda p, a = rr / (p . q), x += a p,
// r -= a q, p = r + (rr'/rr) p; counts the anchors still active.  G_m is the sum of the
// nsplit partial products (split_sum).
template <typename Real>
__global__ void __launch_bounds__(32 * kAncWarps) k_anc_cg(Params p, int nrc, int rows_per_chunk,
                                                           dev::Band band, int nsplit,
                                                           const Real *A, const Real *G,
                                                           const double *part, const Real *S,
                                                           Anchor *st, Real *x, Real *r,
                                                           Real *pv, Real *q, int *active)
{
    const int lane = threadIdx.x & 31;
    const int m = blockIdx.x * kAncWarps + (threadIdx.x >> 5);
    if (m >= p.M) return;
    Anchor &a = st[m];
    if (a.done) return;
    double cs[1] = {0.0};   // sum_j T_jm: lane-strided row chunks in order, then the warp tree
    for (int c = lane; c < nrc; c += 32) {   // chunks off anchor m's window hold no entry
        const long long j0 = (long long)c * rows_per_chunk;
        if (band.hits(j0, min((long long)p.M, j0 + rows_per_chunk), m, m + 1))
            cs[0] += part[((size_t)c * p.M + m) * 3];
    }
    warp_sums(cs);
    const size_t o = (size_t)m * p.ld, split = (size_t)p.M * p.ld;
    const double rr = a.rr;
    const Real csr = (Real)cs[0], spr = (Real)a.sp, lamr = (Real)a.lam;
    Real pq[1] = {Real(0)};
    for (int i = lane; i < p.ld; i += 32) {
        const Real g = split_sum(G, split, o + i, nsplit);
        const Real qi = g - csr * A[o + i] - S[o + i] * spr + lamr * pv[o + i];
        q[o + i] = qi;
        pq[0] += pv[o + i] * qi;
    }
    warp_sums(pq);
    const double pqd = (double)pq[0];
    if (!(pqd > 0.0) || !isfinite(pqd)) {
        if (lane == 0) {
            a.done = 1;
            if (!(rr <= p.cg_tol2 * a.rhs2)) a.status = FBSDE_ERR_CG;
        }
        return;
    }
    const double step = rr / pqd;
    const Real stepr = (Real)step;
    Real rn[1] = {Real(0)};
    for (int i = lane; i < p.ld; i += 32) {
        x[o + i] += stepr * pv[o + i];
        const Real ri = r[o + i] - stepr * q[o + i];
        r[o + i] = ri;
        rn[0] += ri * ri;
    }
    warp_sums(rn);
    const double rr_new = (double)rn[0], beta = rr_new / rr;
    const Real betar = (Real)beta;
    Real b[2] = {Real(0), Real(0)};
    for (int i = lane; i < p.ld; i += 32) {
        const Real pi = r[o + i] + betar * pv[o + i];
        pv[o + i] = pi;
        b[0] += S[o + i] * pi;
        b[1] += A[o + i] * pi;
    }
    warp_sums(b);
    if (lane == 0) {
        a.rr = rr_new;
        a.sp = (double)b[0];
        a.ap = (double)b[1];
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

// Sums of NV values over the nw warps of a block (warp trees, then the warps in order);
// every thread gets the totals.  sm: this reduction's own [8][NV] slots, so consecutive
// reductions need no barrier between them.
template <typename T, int NV>
__device__ __forceinline__ void block_sums(T (&v)[NV], T (*sm)[NV], int warp, int lane, int nw)
{
    warp_sums(v);
    if (nw == 1) return;
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < NV; ++i) sm[warp][i] = v[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        T s = sm[0][i];
        for (int w = 1; w < nw; ++w) s += sm[w][i];
        v[i] = s;
    }
}

// The CG pass of k_anc_cg with the anchor's vectors in registers: one block of nw <= 8 warps
// per anchor, thread t holding the 16-byte chunks t, t + 32 nw, .. (at most C of them).
// The first phase loads G's splits, A, S, p, r and x together; q stays in registers, and
// the later phases read only S and A again, so a pass moves each vector about once.
// Rows of at most 256 C chunks (the host falls back to k_anc_cg beyond that).
template <typename Real, int C>
__global__ void __launch_bounds__(256) k_anc_cg_reg(Params p, int nrc, int rows_per_chunk,
                                                    dev::Band band, int nsplit, const Real *A,
                                                    const Real *G, const double *part,
                                                    const Real *S, Anchor *st, Real *x, Real *r,
                                                    Real *pv, int *active)
{
    constexpr int E = Chunk<Real>::E;
    __shared__ Real red_pq[8][1], red_rn[8][1], red_b[8][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int m = blockIdx.x;
    Anchor &a = st[m];
    if (a.done) return;   // the whole block
    double cs[1] = {0.0};   // sum_j T_jm, as in k_anc_cg (every warp the same sum)
    for (int c = lane; c < nrc; c += 32) {
        const long long j0 = (long long)c * rows_per_chunk;
        if (band.hits(j0, min((long long)p.M, j0 + rows_per_chunk), m, m + 1))
            cs[0] += part[((size_t)c * p.M + m) * 3];
    }
    warp_sums(cs);
    const int nchk = p.ld / E;
    const size_t o = (size_t)m * p.ld, split = (size_t)p.M * p.ld;
    const double rr = a.rr;
    const Real csr = (Real)cs[0], spr = (Real)a.sp, lamr = (Real)a.lam;
    Chunk<Real> pc[C], qc[C], rc[C], xc[C];
#pragma unroll
    for (int v = 0; v < C; ++v) {
        zero(pc[v]);
        zero(qc[v]);
        zero(rc[v]);
        zero(xc[v]);
    }
    // G_m: the splits added in z order (split_sum's order), C independent loads per split
    for (int z = 0; z < nsplit; ++z) {
#pragma unroll
        for (int v = 0; v < C; ++v) {
            const int ci = threadIdx.x + blockDim.x * v;
            if (ci < nchk) {
                const Chunk<Real> t = dev::ldg_chunk(G + z * split + o + (size_t)ci * E);
#pragma unroll
                for (int e = 0; e < E; ++e) qc[v].v[e] += t.v[e];
            }
        }
    }
    Real pq[1] = {Real(0)};
#pragma unroll
    for (int v = 0; v < C; ++v) {
        const int ci = threadIdx.x + blockDim.x * v;
        if (ci < nchk) {
            const size_t ix = o + (size_t)ci * E;
            const Chunk<Real> ac = dev::ldg_chunk(A + ix), sc = dev::ldg_chunk(S + ix);
            pc[v] = dev::ld_chunk(pv + ix);
            rc[v] = dev::ld_chunk(r + ix);
            xc[v] = dev::ld_chunk(x + ix);
#pragma unroll
            for (int e = 0; e < E; ++e) {
                qc[v].v[e] = qc[v].v[e] - csr * ac.v[e] - sc.v[e] * spr + lamr * pc[v].v[e];
                pq[0] += pc[v].v[e] * qc[v].v[e];
            }
        }
    }
    block_sums(pq, red_pq, warp, lane, nw);
    const double pqd = (double)pq[0];
    if (!(pqd > 0.0) || !isfinite(pqd)) {   // the same value in every thread
        if (threadIdx.x == 0) {
            a.done = 1;
            if (!(rr <= p.cg_tol2 * a.rhs2)) a.status = FBSDE_ERR_CG;
        }
        return;
    }
    const double step = rr / pqd;
    const Real stepr = (Real)step;
    Real rn[1] = {Real(0)};
#pragma unroll
    for (int v = 0; v < C; ++v) {
        const int ci = threadIdx.x + blockDim.x * v;
        if (ci < nchk) {
            const size_t ix = o + (size_t)ci * E;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                xc[v].v[e] += stepr * pc[v].v[e];
                rc[v].v[e] = rc[v].v[e] - stepr * qc[v].v[e];
                rn[0] += rc[v].v[e] * rc[v].v[e];
            }
            dev::st_chunk(x + ix, xc[v]);
            dev::st_chunk(r + ix, rc[v]);
        }
    }
    block_sums(rn, red_rn, warp, lane, nw);
    const double rr_new = (double)rn[0], beta = rr_new / rr;
    const Real betar = (Real)beta;
    Real b[2] = {Real(0), Real(0)};
#pragma unroll
    for (int v = 0; v < C; ++v) {
        const int ci = threadIdx.x + blockDim.x * v;
        if (ci < nchk) {
            const size_t ix = o + (size_t)ci * E;
            const Chunk<Real> ac = dev::ldg_chunk(A + ix), sc = dev::ldg_chunk(S + ix);
#pragma unroll
            for (int e = 0; e < E; ++e) {
                pc[v].v[e] = rc[v].v[e] + betar * pc[v].v[e];
                b[0] += sc.v[e] * pc[v].v[e];
                b[1] += ac.v[e] * pc[v].v[e];
            }
            dev::st_chunk(pv + ix, pc[v]);
        }
    }
    block_sums(b, red_b, warp, lane, nw);
    if (threadIdx.x == 0) {
        a.rr = rr_new;
        a.sp = (double)b[0];
        a.ap = (double)b[1];
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

// Direct solve of each anchor's regression over its batch (the batch reading of Remark
// 2.1), in place of the CG passes: one block per anchor m, of one thread per tile with
// TPT = 1 (rounded up to whole warps), of kDirThreads threads with TPT = 2.
//   1. The weighted second moment of the window, sum_q w_jm D_j D_j^T with D_j = P_j - A_m
//      over j = (m + q) mod M, q < Kb, summed over q in order in the stream precision: the
//      lower triangle in 8 x 4 tiles (rows 8 I.., columns 4 K.., 4 K <= 8 I + 7), at most
//      TPT tiles in registers per thread (TPT = 1 while the triangle has at most
//      kDirThreads tiles, d <= 120); the window's rows pass through shared
//      memory kDirRows at a time (one warp per row), padded with zeros to a multiple of 8.
//   2. Gamma_m + lambda_m I = moment / W_m - S_m S_m^T + lambda_m I, the operator of the
//      CG pass (Eq. 3.19's), in the same registers.
//   3. Its LDL^T factorisation, right-looking on the registers with one barrier per column
//      (the column passes through shared memory, where it stays as the factor; the
//      operator is symmetric positive definite for lambda_m > 0, so no pivoting), then
//      L y = rhs, D z = y, L^T x = z by one warp with the vector in registers.
// The entry point requires ridge_rel > 0, so every pivot is at least lambda_m in exact
// arithmetic; a pivot that is still not positive and finite leaves x = 0 and the anchor's
// status FBSDE_ERR_CG.  Anchors whose right-hand side is zero (done after the setup) keep
// x = 0.
constexpr int kDirThreads = 256, kDirRows = 32, kDirMaxD = 128;
// Padded length of a row (and pitch of the factor's columns): a multiple of 8.
__host__ __device__ inline int dir_pad(int d) { return (d + 7) / 8 * 8; }
inline size_t dir_smem_bytes(int d, size_t rs)
{
    const size_t dp = (size_t)dir_pad(d);
    const size_t fac = (size_t)d * dp + dp;    // the factor's columns, S_m
    const size_t rows = 2 * (size_t)kDirRows * dp;   // w D and D of the rows
    return std::max(fac, rows) * rs;
}
template <typename Real> struct Vec4;
template <> struct Vec4<float> {
    static __device__ __forceinline__ void ld(float (&v)[4], const float *q)
    {
        const float4 t = *reinterpret_cast<const float4 *>(q);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
};
template <> struct Vec4<double> {
    static __device__ __forceinline__ void ld(double (&v)[4], const double *q)
    {
        const double2 a = *reinterpret_cast<const double2 *>(q);
        const double2 b = *reinterpret_cast<const double2 *>(q + 2);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
};
template <typename Real, int TPT>
__global__ void __launch_bounds__(kDirThreads) k_anc_direct(Params p, long long Kb,
                                                             const Real *P, const Real *A,
                                                             const Real *W, const Real *S,
                                                             const Real *rhs, Anchor *st,
                                                             Real *x)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    Real *G = reinterpret_cast<Real *>(dsm);
    const int m = blockIdx.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int d = p.d, ld = p.ld, dp = dir_pad(d);
    Anchor &a = st[m];
    if (a.done) return;   // the whole block
    const size_t o = (size_t)m * ld;
    const int nI = dp / 8, nK = dp / 4;
    // the thread's tiles, tile b counted along the rows of tiles: row I holds
    // min(2 I + 2, nK) tiles
    int ti[TPT], tk[TPT];
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
        int b = t + (int)blockDim.x * u;
        ti[u] = -1;
        tk[u] = 0;
        for (int I = 0; I < nI; ++I) {
            const int n = min(2 * I + 2, nK);
            if (b < n) {
                ti[u] = I;
                tk[u] = b;
                break;
            }
            b -= n;
        }
    }
    Real acc[TPT][8][4];
#pragma unroll
    for (int u = 0; u < TPT; ++u)
#pragma unroll
        for (int ii = 0; ii < 8; ++ii)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) acc[u][ii][kk] = Real(0);
    Real *Dw = G, *Dr = G + (size_t)kDirRows * dp;   // the rows: w D and D
    for (long long q0 = 0; q0 < Kb; q0 += kDirRows) {
        const int nr = (int)min((long long)kDirRows, Kb - q0);
        __syncthreads();   // the previous rows are used up
        for (int r = warp; r < nr; r += (int)(blockDim.x >> 5)) {
            long long j = m + q0 + r;
            if (j >= p.M) j -= p.M;
            const Real w = W[(size_t)j * p.M + m];
            const Real *pj = P + (size_t)j * ld;
            for (int i = lane; i < dp; i += 32) {
                const Real dv = i < d ? pj[i] - A[o + i] : Real(0);
                Dr[r * dp + i] = dv;
                Dw[r * dp + i] = w * dv;
            }
        }
        __syncthreads();
        for (int r = 0; r < nr; ++r) {
#pragma unroll
            for (int u = 0; u < TPT; ++u) {
                if (ti[u] < 0) continue;
                Real wi[8], dk[4];
                Vec4<Real>::ld(*reinterpret_cast<Real(*)[4]>(wi), Dw + r * dp + 8 * ti[u]);
                Vec4<Real>::ld(*reinterpret_cast<Real(*)[4]>(wi + 4), Dw + r * dp + 8 * ti[u] + 4);
                Vec4<Real>::ld(dk, Dr + r * dp + 4 * tk[u]);
#pragma unroll
                for (int ii = 0; ii < 8; ++ii)
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) acc[u][ii][kk] += wi[ii] * dk[kk];
            }
        }
    }
    __syncthreads();   // the row buffers become the factor's columns
    Real *Lc = G;                          // column c of the factor at Lc[c * dp + i], i >= c
    Real *Sv = G + (size_t)d * dp;         // S_m
    for (int e = t; e < d * dp; e += blockDim.x) Lc[e] = Real(0);   // padding stays 0
    for (int i = t; i < d; i += blockDim.x) Sv[i] = S[o + i];
    __syncthreads();
    // Gamma + lambda I in the same registers: entry (8 I + ii, 4 K + kk) of tile u
    const Real invW = (Real)(1.0 / a.W), lam = (Real)a.lam;
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
        if (ti[u] < 0) continue;
#pragma unroll
        for (int ii = 0; ii < 8; ++ii)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const int i = 8 * ti[u] + ii, k = 4 * tk[u] + kk;
                Real g = Real(0);
                if (i < d && k <= i) {
                    g = acc[u][ii][kk] * invW - Sv[i] * Sv[k];
                    if (i == k) g += lam;
                }
                acc[u][ii][kk] = g;
            }
    }
    // LDL^T, right-looking on the registers: before step c the owners of column c (entries
    // (i, c), c <= i < d, every update of the steps before applied) write it to Lc; after
    // the barrier every thread updates its entries (i, k), c < k <= i, by
    // -= Lc[c][i] Lc[c][k] / D_c with D_c = Lc[c][c].  The column's entries above c and
    // beyond d are zero in Lc, so tiles wholly below and right of c need no masks; the
    // entries above the diagonal of a tile that crosses it are never read.
    bool fail = false;
    for (int c = 0; c < d; ++c) {
#pragma unroll
        for (int u = 0; u < TPT; ++u) {
            if (ti[u] < 0 || tk[u] != (c >> 2)) continue;
#pragma unroll
            for (int ii = 0; ii < 8; ++ii) {
                const int i = 8 * ti[u] + ii;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    if ((c & 3) == kk && i >= c && i < d) Lc[c * dp + i] = acc[u][ii][kk];
            }
        }
        __syncthreads();
        const Real piv = Lc[c * dp + c];   // the same value in every thread
        if (!(piv > Real(0)) || !isfinite(piv)) {
            fail = true;
            break;
        }
        const Real ip = Real(1) / piv;
#pragma unroll
        for (int u = 0; u < TPT; ++u) {
            if (ti[u] < 0 || 4 * tk[u] + 3 <= c) continue;   // every column of the tile done
            Real li[8], lk[4];
            Vec4<Real>::ld(*reinterpret_cast<Real(*)[4]>(li), Lc + c * dp + 8 * ti[u]);
            Vec4<Real>::ld(*reinterpret_cast<Real(*)[4]>(li + 4), Lc + c * dp + 8 * ti[u] + 4);
            Vec4<Real>::ld(lk, Lc + c * dp + 4 * tk[u]);
            if (4 * tk[u] <= c) {   // the tile holds column c: only its columns k > c move
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    if (4 * tk[u] + kk <= c) lk[kk] = Real(0);
            }
            // rows i <= c hold entries above the diagonal or finished ones: the column's
            // entry there is Lc[c][i], zero above c and D_c at c
            if (8 * ti[u] <= c) {
#pragma unroll
                for (int ii = 0; ii < 8; ++ii)
                    if (8 * ti[u] + ii <= c) li[ii] = Real(0);
            }
#pragma unroll
            for (int ii = 0; ii < 8; ++ii) {
                const Real l = li[ii] * ip;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) acc[u][ii][kk] -= l * lk[kk];
            }
        }
    }
    if (t >= 32) return;
    if (fail) {
        if (lane == 0) {
            a.status = FBSDE_ERR_CG;
            a.done = 1;
        }
        return;   // x stays 0 from the setup
    }
    // L y = rhs, z = D^{-1} y, L^T x = z with L_ic = Lc[c][i] / D_c; lane l holds the
    // entries l, l + 32, l + 64, l + 96 of y (then z, then x) in registers
    constexpr int kV = kDirMaxD / 32;
    Real yv[kV], invD[kV];
#pragma unroll
    for (int v = 0; v < kV; ++v) {
        const int i = lane + 32 * v;
        yv[v] = i < d ? rhs[o + i] : Real(0);
        invD[v] = i < d ? Real(1) / Lc[i * dp + i] : Real(0);
    }
    for (int c = 0; c < d; ++c) {
        Real yc = Real(0);
#pragma unroll
        for (int v = 0; v < kV; ++v)
            if ((c >> 5) == v) yc = __shfl_sync(0xffffffffu, yv[v] * invD[v], c & 31);
#pragma unroll
        for (int v = 0; v < kV; ++v) {
            const int i = lane + 32 * v;
            if (i > c && i < d) yv[v] -= Lc[c * dp + i] * yc;
        }
    }
#pragma unroll
    for (int v = 0; v < kV; ++v) yv[v] *= invD[v];
    for (int c = d - 1; c > 0; --c) {   // x_c is final once the entries below are in
        Real xc = Real(0);
#pragma unroll
        for (int v = 0; v < kV; ++v)
            if ((c >> 5) == v) xc = __shfl_sync(0xffffffffu, yv[v], c & 31);
#pragma unroll
        for (int v = 0; v < kV; ++v) {
            const int k = lane + 32 * v;
            if (k < c) yv[v] -= Lc[k * dp + c] * invD[v] * xc;
        }
    }
#pragma unroll
    for (int v = 0; v < kV; ++v) {
        const int i = lane + 32 * v;
        if (i < d) x[o + i] = yv[v];
    }
}

// Per anchor: alpha = c - S . x (Eq. 3.20), Z = sigma x, the features of f at
// (t_k, X_k^m, Z) and Newton (2.16)-(2.17) for Y_k^m (lane 0).
template <typename Real>
__global__ void __launch_bounds__(32 * kAncWarps) k_anc_newton(Params p, double t_k,
                                                               const double *x0, const Real *A,
                                                               const Real *S, const Real *x,
                                                               Anchor *st, double *Ynew,
                                                               int *status)
{
    const int lane = threadIdx.x & 31;
    const int m = blockIdx.x * kAncWarps + (threadIdx.x >> 5);
    if (m >= p.M) return;
    Anchor &a = st[m];
    const size_t o = (size_t)m * p.ld;
    // S . x, sum cos(x0 + A), sum x, |x|^2: lane sums and the warp tree in the stream
    // precision (as the per-anchor vectors themselves), widened once
    Real acc[4] = {Real(0), Real(0), Real(0), Real(0)};
    for (int i = lane; i < p.ld; i += 32) {
        const Real xi = x[o + i];
        acc[0] += S[o + i] * xi;
        if (i < p.d) acc[1] += dev::cos_stream((Real)x0[i] + A[o + i]);
        acc[2] += xi;
        acc[3] += xi * xi;
    }
    warp_sums(acc);
    if (lane == 0) {
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
template <typename Real>
__global__ void __launch_bounds__(256) k_anc_output(int M, int d, const double *Y, const Real *x,
                                                    double *u0, double *grad)
{
    __shared__ double sm[32];
    double acc[1] = {0.0};
    for (int m = threadIdx.x; m < M; m += blockDim.x) acc[0] += Y[m];
    bsum(acc, sm);
    if (threadIdx.x == 0) *u0 = acc[0] / M;
    if (grad)
        for (int i = threadIdx.x; i < d; i += blockDim.x) grad[i] = (double)x[i];
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

struct Lay {
    int d, ld, N;
    int64_t M;
    size_t rs;   // bytes of one stream-precision value
    int nrc, nsplit, kc;   // row chunks of the column pass; K splits (kc rows each) of the
                           // tall contractions
    size_t P, A, YP, G1, W, T, G2, G3, S, rhs, x, r, pv, q, Y, Yn, pn, an, cs, st, cnt, total;
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
    if (P->mu0 != 0.0 || P->mu1 != 0.0 || P->sig1 != 0.0) return false;   // driftless only
    L.d = P->d;
    L.ld = (P->d + 3) / 4 * 4;
    L.N = P->N;
    L.M = P->M;
    L.rs = P->precision == FBSDE_FP32 ? 4 : 8;
    const size_t M = (size_t)L.M, ld = (size_t)L.ld;
    L.nrc = (int)((L.M + kRowChunk - 1) / kRowChunk);
    {   // enough blocks for about two waves of the 152 SMs, at least 128 rows per split
        const long long tiles = ((long long)(ld + 63) / 64) * ((L.M + 63) / 64);
        const long long want = std::max(1ll, (2ll * 152 * 4 + tiles - 1) / tiles);
        const long long ns = std::max(1ll, std::min(want, (long long)(L.M / 128)));
        L.kc = (int)(((L.M + ns - 1) / ns + 15) / 16 * 16);
        L.nsplit = (int)((L.M + L.kc - 1) / L.kc);   // every split holds rows
    }
    size_t o = 0;
    auto take = [&](size_t b) { const size_t r = o; o = up(o + b); return r; };
    L.P = take(M * ld * L.rs);
    L.A = take(M * ld * L.rs);
    L.YP = take(M * ld * L.rs);
    L.G1 = take(M * M * L.rs);
    L.W = take(M * M * L.rs);
    L.T = take(M * M * L.rs);
    L.G2 = take((size_t)L.nsplit * M * ld * L.rs);
    L.G3 = take((size_t)L.nsplit * M * ld * L.rs);
    L.S = take(M * ld * L.rs);
    L.rhs = take(M * ld * L.rs);
    L.x = take(M * ld * L.rs);
    L.r = take(M * ld * L.rs);
    L.pv = take(M * ld * L.rs);
    L.q = take(M * ld * L.rs);
    L.Y = take(M * 8);
    L.Yn = take(M * 8);
    L.pn = take(M * 8);
    L.an = take(M * 8);
    L.cs = take((size_t)L.nrc * M * 3 * 8);
    L.st = take(M * sizeof(Anchor));
    L.cnt = take(4 * sizeof(int));
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

// Epilogue of the CG pass's product U = P V^T on the tensor cores: in place of U, the
// matrix T_jm = w_jm (U_jm - A_m . v_m) / W_m of the next product and its column sums
// over each 128-row tile (k_anc_columns in mode 1, fused; same FP32 arithmetic).  Anchors
// that are done keep their old column of T.
struct TcColumnsEpi {
    const float *W;
    float *T;
    const Anchor *st;
    double *part;
    int M;
    static constexpr bool kColSums = true, kPrefetch = true;
    struct Col {
        float ap, inv;
        int skip;
    };
    struct Pre {
        float w[32];   // W_jm of the 32 rows a warp hands out
    };
    __device__ __forceinline__ void prefetch(int j0, int m, const Col &, Pre &pr) const
    {
#pragma unroll
        for (int rr = 0; rr < 32; ++rr)
            pr.w[rr] = (m >= 0 && j0 + rr < M) ? W[(size_t)(j0 + rr) * M + m] : 0.0f;
    }
    __device__ __forceinline__ Col column(int m) const
    {
        Col c{0.0f, 0.0f, 1};
        if (m >= 0) {
            const Anchor &a = st[m];
            c.skip = a.done;
            c.ap = (float)a.ap;
            c.inv = (float)(1.0 / a.W);
        }
        return c;
    }
    __device__ __forceinline__ float put(int, int j, int m, float u, const Col &c, const Pre &pr,
                                         int rr) const
    {
        if (c.skip) return 0.0f;
        const float t = pr.w[rr] * (u - c.ap) * c.inv;
        T[(size_t)j * M + m] = t;
        return t;
    }
    __device__ __forceinline__ void colsum(int tile, int m, float s) const
    {
        part[((size_t)tile * M + m) * 3] = (double)s;
    }
};

// The FP32 products of M >= 1024 particles go to the tensor cores (k_gemm_tc, split
// TF32); the k-contiguous layout there needs 16-byte rows and k ranges in steps of 4.
inline bool tc_layout_ok(bool tn, int K, int kc, const void *A, int lda, const void *B, int ldb)
{
    if (tn) return true;
    return K % 4 == 0 && kc % 4 == 0 && lda % 4 == 0 && ldb % 4 == 0 &&
           reinterpret_cast<uintptr_t>(A) % 16 == 0 && reinterpret_cast<uintptr_t>(B) % 16 == 0;
}

template <bool TN, class Epi>
cudaError_t gemm_tc(int Mr, int Nc, int K, int kc, const float *A, int lda, const float *B,
                    int ldb, const Epi &epi, int *status, cudaStream_t s, dev::Band band)
{
    cudaError_t e = cudaFuncSetAttribute(dev::k_gemm_tc<TN, Epi>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)dev::kTcSmemBytes);
    if (e != cudaSuccess) return e;
    const dim3 grid((Nc + dev::kTcBN - 1) / dev::kTcBN, (Mr + dev::kTcBM - 1) / dev::kTcBM,
                    (K + kc - 1) / kc);
    dev::k_gemm_tc<TN, Epi><<<grid, dev::kTcThreads, dev::kTcSmemBytes, s>>>(Mr, Nc, K, kc, A, lda,
                                                                           B, ldb, epi, status,
                                                                           band);
    return cudaGetLastError();
}

template <typename Real, bool TN>
cudaError_t gemm(int Mr, int Nc, int K, int kc, const Real *A, int lda, const Real *B, int ldb,
                 Real *C, int ldc, int *status, cudaStream_t s, dev::Band band)
{
    if constexpr (sizeof(Real) == 4) {
        if (Mr >= 1024 && tc_layout_ok(TN, K, kc, A, lda, B, ldb))
            return gemm_tc<TN>(Mr, Nc, K, kc, A, lda, B, ldb, dev::TcStore{C, Mr, ldc}, status, s,
                               band);
    }
    const dim3 grid((Nc + 63) / 64, (Mr + 63) / 64, (K + kc - 1) / kc);
    k_gemm<Real, TN><<<grid, 256, 0, s>>>(Mr, Nc, K, kc, A, lda, B, ldb, C, ldc, band);
    return cudaGetLastError();
}

#define ANC_TRY(call)                                                                       \
    do {                                                                                     \
        if ((e = (call)) != cudaSuccess) return e;                                           \
    } while (0)

// Loop control of a level's per-anchor CG, a conditional while node of a CUDA graph.
// cnt: [0] anchors that iterated on in the last pass (k_anc_cg counts them), [1] device
// status, [2] passes of the current loop, [3] passes of the whole call.
__global__ void k_anc_loop_reset(int *cnt, cudaGraphConditionalHandle h)
{
    if (threadIdx.x != 0) return;
    cnt[0] = 0;
    cnt[2] = 0;
    cudaGraphSetConditional(h, 1u);
}

// After a pass: go on while some anchor is still iterating and fewer than max_iter passes
// ran.
__global__ void k_anc_loop_next(int *cnt, int max_iter, cudaGraphConditionalHandle h)
{
    if (threadIdx.x != 0) return;
    const int active = cnt[0], passes = cnt[2] + 1;
    cnt[0] = 0;
    cnt[2] = passes;
    cnt[3] += 1;
    cudaGraphSetConditional(h, (active > 0 && passes < max_iter) ? 1u : 0u);
}

// Block of the register-resident CG pass for rows of nchk 16-byte chunks: nw warps and C
// chunks per thread with 32 nw C >= nchk, C in {1, 2, 4} and nw <= 8 (C = 0: rows longer
// than 1024 chunks, which take the streaming k_anc_cg).
struct CgShape {
    int nw, C;
};
CgShape cg_shape(int nchk)
{
    if (nchk > 32 * 8 * 4) return {0, 0};
    const int nw = std::min(8, (nchk + 127) / 128);
    const int per = (nchk + 32 * nw - 1) / (32 * nw);
    return {nw, per <= 1 ? 1 : per <= 2 ? 2 : 4};
}

// One query, enqueued on s, which must be capturing into a CUDA graph: the forward sweep,
// then the levels k = N-1..0, each level's CG passes as a conditional while node whose
// body is captured on the stream b.  The device status accumulates in cnt[1].
// Kb: particles per anchor's regression (the cyclic window; Kb = M: all of them).
template <typename Real>
cudaError_t emit_one(const fbsde_problem *Pb, const Lay &L, const double *x0, uint64_t seed,
                     uint32_t sidx, double *u0, double *grad, char *ws, cudaStream_t s,
                     cudaStream_t b, long long Kb, bool direct)
{
    cudaError_t e;
    Params p = params_of(Pb, L, seed);
    const int M = (int)L.M, ld = L.ld;
    Real *P = reinterpret_cast<Real *>(ws + L.P), *A = reinterpret_cast<Real *>(ws + L.A);
    Real *YP = reinterpret_cast<Real *>(ws + L.YP);
    Real *G1 = reinterpret_cast<Real *>(ws + L.G1), *W = reinterpret_cast<Real *>(ws + L.W);
    Real *T = reinterpret_cast<Real *>(ws + L.T);
    Real *G2 = reinterpret_cast<Real *>(ws + L.G2), *G3 = reinterpret_cast<Real *>(ws + L.G3);
    Real *S = reinterpret_cast<Real *>(ws + L.S), *rhs = reinterpret_cast<Real *>(ws + L.rhs);
    Real *x = reinterpret_cast<Real *>(ws + L.x), *r = reinterpret_cast<Real *>(ws + L.r);
    Real *pv = reinterpret_cast<Real *>(ws + L.pv), *q = reinterpret_cast<Real *>(ws + L.q);
    double *Y = reinterpret_cast<double *>(ws + L.Y), *Yn = reinterpret_cast<double *>(ws + L.Yn);
    double *pn = reinterpret_cast<double *>(ws + L.pn), *an = reinterpret_cast<double *>(ws + L.an);
    double *cs = reinterpret_cast<double *>(ws + L.cs);
    Anchor *st = reinterpret_cast<Anchor *>(ws + L.st);
    int *cnt = reinterpret_cast<int *>(ws + L.cnt);
    k_anc_terminal<Real><<<M, 128, 0, s>>>(p, x0, sidx, P, Y);
    ANC_TRY(cudaGetLastError());
    const dim3 cgrid((M + 127) / 128, L.nrc);
    const int awarps = (M + kAncWarps - 1) / kAncWarps;   // blocks of the per-anchor kernels
    // FP32 with M >= 1024: the CG pass's column pass runs in the tensor-core product's
    // epilogue, with column sums over 128-row tiles
    const bool fused = sizeof(Real) == 4 && M >= 1024 && tc_layout_ok(false, ld, ld, P, ld, A, ld);
    const int nrc_fused = (M + dev::kTcBM - 1) / dev::kTcBM;
    // batch reading: the products cover only the band of entries the windows use (tiles and
    // K-splits off it are skipped); T's entries off the band stay zero for the whole solve
    const dev::Band band{(long long)M, Kb < M ? Kb : (long long)M};
    if (fused && Kb < M && !direct)
        ANC_TRY(cudaMemsetAsync(T, 0, (size_t)M * M * sizeof(Real), s));
    // direct batch solve: one 8 x 4 tile per thread while the triangle has at most
    // kDirThreads of them (fewer registers and threads, more blocks per SM), else two
    const size_t dir_smem = dir_smem_bytes(L.d, sizeof(Real));
    const int dir_nI = dir_pad(L.d) / 8;
    const bool dir_two = dir_nI * (dir_nI + 1) > kDirThreads;
    if (direct)
        ANC_TRY(cudaFuncSetAttribute(dir_two ? k_anc_direct<Real, 2> : k_anc_direct<Real, 1>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dir_smem));
    const CgShape cg = cg_shape(ld / Chunk<Real>::E);
    for (int k = L.N - 1; k >= 0; --k) {
        const double t_k = k * p.dt;
        const double a = (double)k / (double)(k + 1), bb = p.sigma * std::sqrt(p.dt * a);
        k_anc_step<Real><<<152 * 8, 256, 0, s>>>(p, k, sidx, a, bb, P, A);
        ANC_TRY(cudaGetLastError());
        k_anc_rows<Real><<<M, 128, 0, s>>>(p, P, A, Y, pn, an, YP);
        ANC_TRY(cudaGetLastError());
        ANC_TRY((gemm<Real, false>(M, M, ld, ld, P, ld, A, ld, G1, M, cnt + 1, s, band)));   // P A^T
        const double rho_ref = p.sigma * p.sigma * p.d * (t_k + (k + 1) * p.dt);
        k_anc_columns<Real><<<cgrid, 128, 0, s>>>(p, 0, rho_ref, Kb, G1, pn, an, Y, W, T, st, cs);
        ANC_TRY(cudaGetLastError());
        ANC_TRY((gemm<Real, true>(M, ld, M, L.kc, W, M, P, ld, G2, ld, cnt + 1, s, band)));    // W^T P
        ANC_TRY((gemm<Real, true>(M, ld, M, L.kc, W, M, YP, ld, G3, ld, cnt + 1, s, band)));   // W^T (Y P)
        k_anc_setup<Real><<<awarps, 32 * kAncWarps, 0, s>>>(p, L.nrc, L.nsplit, A, G2, G3, cs, st, S,
                                                           rhs, x, r, pv);
        ANC_TRY(cudaGetLastError());
        // the CG passes: a conditional while node (body on b) that repeats while some anchor
        // iterates on and fewer than cg_max_iter passes ran; or each anchor's direct solve
        if (direct) {
            if (dir_two)
                k_anc_direct<Real, 2><<<M, kDirThreads, dir_smem, s>>>(p, band.Kb, P, A, W, S, rhs,
                                                                       st, x);
            else
                k_anc_direct<Real, 1><<<M, 32 * ((dir_nI * (dir_nI + 1) + 31) / 32), dir_smem, s>>>(
                    p, band.Kb, P, A, W, S, rhs, st, x);
            ANC_TRY(cudaGetLastError());
        } else {
            cudaStreamCaptureStatus cst;
            cudaGraph_t g = nullptr;
            const cudaGraphNode_t *deps = nullptr;
            const cudaGraphEdgeData *ed = nullptr;
            size_t nd = 0;
            ANC_TRY(cudaStreamGetCaptureInfo(s, &cst, nullptr, &g, &deps, &ed, &nd));
            if (cst != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
            cudaGraphConditionalHandle h;
            ANC_TRY(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
            k_anc_loop_reset<<<1, 32, 0, s>>>(cnt, h);
            ANC_TRY(cudaGetLastError());
            ANC_TRY(cudaStreamGetCaptureInfo(s, &cst, nullptr, &g, &deps, &ed, &nd));
            cudaGraphNodeParams np = {};
            np.type = cudaGraphNodeTypeConditional;
            np.conditional.handle = h;
            np.conditional.type = cudaGraphCondTypeWhile;
            np.conditional.size = 1;
            cudaGraphNode_t node;
            ANC_TRY(cudaGraphAddNode(&node, g, deps, ed, nd, &np));
            ANC_TRY(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1,
                                                        cudaStreamSetCaptureDependencies));
            ANC_TRY(cudaStreamBeginCaptureToGraph(b, np.conditional.phGraph_out[0], nullptr, nullptr,
                                                  0, cudaStreamCaptureModeRelaxed));
            cudaError_t eb = cudaSuccess;
            if (fused) {   // T and its column sums straight from the product's epilogue
                if constexpr (sizeof(Real) == 4)
                    eb = gemm_tc<false>(M, M, ld, ld, P, ld, pv, ld, TcColumnsEpi{W, T, st, cs, M},
                                        cnt + 1, b, band);
            } else {
                eb = gemm<Real, false>(M, M, ld, ld, P, ld, pv, ld, G1, M, cnt + 1, b, band);   // U = P V^T
                if (eb == cudaSuccess) {
                    k_anc_columns<Real><<<cgrid, 128, 0, b>>>(p, 1, 0.0, Kb, G1, pn, an, Y, W, T, st, cs);
                    eb = cudaGetLastError();
                }
            }
            if (eb == cudaSuccess)
                eb = gemm<Real, true>(M, ld, M, L.kc, T, M, P, ld, G2, ld, cnt + 1, b, band);   // T^T P
            if (eb == cudaSuccess) {
                const int nrc_cg = fused ? nrc_fused : L.nrc;
                const int rpc = fused ? dev::kTcBM : kRowChunk;
                switch (cg.C) {
                case 1:
                    k_anc_cg_reg<Real, 1><<<M, 32 * cg.nw, 0, b>>>(p, nrc_cg, rpc, band, L.nsplit,
                                                                   A, G2, cs, S, st, x, r, pv, cnt);
                    break;
                case 2:
                    k_anc_cg_reg<Real, 2><<<M, 32 * cg.nw, 0, b>>>(p, nrc_cg, rpc, band, L.nsplit,
                                                                   A, G2, cs, S, st, x, r, pv, cnt);
                    break;
                case 4:
                    k_anc_cg_reg<Real, 4><<<M, 32 * cg.nw, 0, b>>>(p, nrc_cg, rpc, band, L.nsplit,
                                                                   A, G2, cs, S, st, x, r, pv, cnt);
                    break;
                default:
                    k_anc_cg<Real><<<awarps, 32 * kAncWarps, 0, b>>>(p, nrc_cg, rpc, band, L.nsplit,
                                                                     A, G2, cs, S, st, x, r, pv, q,
                                                                     cnt);
                }
                eb = cudaGetLastError();
            }
            if (eb == cudaSuccess) {
                k_anc_loop_next<<<1, 32, 0, b>>>(cnt, p.cg_max_iter, h);
                eb = cudaGetLastError();
            }
            cudaGraph_t ended = nullptr;
            const cudaError_t ee = cudaStreamEndCapture(b, &ended);
            if (eb != cudaSuccess) return eb;
            if (ee != cudaSuccess) return ee;
        }
        k_anc_newton<Real><<<awarps, 32 * kAncWarps, 0, s>>>(p, t_k, x0, A, S, x, st, Yn, cnt + 1);
        ANC_TRY(cudaGetLastError());
        std::swap(P, A);   // level k's rows are the cloud of level k-1
        std::swap(Y, Yn);
    }
    k_anc_output<Real><<<1, 256, 0, s>>>(M, L.d, Y, x, u0, grad);
    return cudaGetLastError();
}

// Every query of a call, enqueued on the capturing stream s (bodies on b): the counters and
// the status word are cleared once, then the queries run one after the other on the
// shared workspace.
cudaError_t emit_call(const fbsde_problem *P, const Lay &L, int64_t K, bool direct, int32_t Q,
                      const double *x0, uint64_t seed, uint32_t solve_index0, double *u0,
                      double *grad_u0, char *ws, cudaStream_t s, cudaStream_t b)
{
    cudaError_t e;
    ANC_TRY(cudaMemsetAsync(ws + L.cnt, 0, 4 * sizeof(int), s));
    for (int q = 0; q < Q; ++q) {
        const double *xq = x0 + (size_t)q * P->d;
        double *gq = grad_u0 ? grad_u0 + (size_t)q * P->d : nullptr;
        e = P->precision == FBSDE_FP32
                ? emit_one<float>(P, L, xq, seed, solve_index0 + q, u0 + q, gq, ws, s, b, K, direct)
                : emit_one<double>(P, L, xq, seed, solve_index0 + q, u0 + q, gq, ws, s, b, K,
                                   direct);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Instantiated graphs of whole calls, keyed by device and the bytes of every argument (an
// eager call with the same arguments replays its graph).  Least-recently used entries beyond
// kAncCacheSize are destroyed once their last launch has completed; the cache is never
// freed, so no CUDA call runs from a static destructor at process exit.
constexpr size_t kAncCacheSize = 8;
struct AncGraph {
    int dev;
    std::vector<unsigned char> key;
    cudaGraphExec_t exec;
    cudaEvent_t last;
};
struct AncCache {
    std::mutex mu;
    std::list<AncGraph> lru;
    cudaStream_t cap[64] = {}, body[64] = {};
};
AncCache *g_anc = new AncCache();

template <typename T> void put(std::vector<unsigned char> &k, const T &v)
{
    const unsigned char *b = reinterpret_cast<const unsigned char *>(&v);
    k.insert(k.end(), b, b + sizeof(T));
}

cudaError_t launch_call(const fbsde_problem *P, const Lay &L, int64_t K, bool direct, int32_t Q,
                        const double *x0, uint64_t seed, uint32_t solve_index0, double *u0,
                        double *grad_u0, char *ws, cudaStream_t s)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_anc->mu);
    if (!g_anc->cap[dev]) {
        if ((e = cudaStreamCreateWithFlags(&g_anc->cap[dev], cudaStreamNonBlocking)) != cudaSuccess)
            return e;
        if ((e = cudaStreamCreateWithFlags(&g_anc->body[dev], cudaStreamNonBlocking)) != cudaSuccess)
            return e;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if ((e = cudaStreamIsCapturing(s, &cs)) != cudaSuccess) return e;
    if (cs == cudaStreamCaptureStatusActive)   // the caller is capturing: become part of it
        return emit_call(P, L, K, direct, Q, x0, seed, solve_index0, u0, grad_u0, ws, s,
                         g_anc->body[dev]);
    std::vector<unsigned char> key;
    put(key, *P);
    put(key, K);
    put(key, direct);
    put(key, Q);
    put(key, x0);
    put(key, seed);
    put(key, solve_index0);
    put(key, u0);
    put(key, grad_u0);
    put(key, ws);
    auto it = g_anc->lru.begin();
    for (; it != g_anc->lru.end(); ++it)
        if (it->dev == dev && it->key == key) break;
    if (it == g_anc->lru.end()) {
        cudaStream_t c = g_anc->cap[dev];
        if ((e = cudaStreamBeginCapture(c, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
        const cudaError_t ec =
            emit_call(P, L, K, direct, Q, x0, seed, solve_index0, u0, grad_u0, ws, c,
                      g_anc->body[dev]);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(c, &g);
        if (ec != cudaSuccess || e != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            return ec != cudaSuccess ? ec : (e != cudaSuccess ? e : cudaErrorUnknown);
        }
        AncGraph a{dev, key, nullptr, nullptr};
        e = cudaGraphInstantiate(&a.exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&a.last, cudaEventDisableTiming)) != cudaSuccess) {
            cudaGraphExecDestroy(a.exec);
            return e;
        }
        g_anc->lru.push_front(a);
        while (g_anc->lru.size() > kAncCacheSize) {
            AncGraph &old = g_anc->lru.back();
            cudaEventSynchronize(old.last);
            cudaGraphExecDestroy(old.exec);
            cudaEventDestroy(old.last);
            g_anc->lru.pop_back();
        }
        it = g_anc->lru.begin();
    } else if (it != g_anc->lru.begin()) {
        g_anc->lru.splice(g_anc->lru.begin(), g_anc->lru, it);
        it = g_anc->lru.begin();
    }
    if ((e = cudaGraphLaunch(it->exec, s)) != cudaSuccess) return e;
    return cudaEventRecord(it->last, s);
}

// fbsde_solve_batch and fbsde_solve_batch_direct: argument checks, then the call's graph.
int solve_batch(const fbsde_problem *P, int64_t K, bool direct, int32_t Q, const double *x0,
                uint64_t seed, uint32_t solve_index0, double *u0, double *grad_u0,
                void *workspace, size_t workspace_bytes, fbsde_stream_t stream)
{
    Lay L;
    if (!lay(P, L) || Q < 1 || !x0 || !u0) return FBSDE_ERR_ARG;
    if (K < 2 || K > L.M) return FBSDE_ERR_ARG;
    // the direct factorisation needs a positive ridge: it bounds every pivot below by lambda_m
    if (direct && (P->d > kDirMaxD || !(P->ridge_rel > 0.0))) return FBSDE_ERR_ARG;
    if ((P->kind == FBSDE_HJB_LOGQUAD || P->kind == FBSDE_AFFINE_TEST) && !P->theta)
        return FBSDE_ERR_ARG;
    if (!workspace || workspace_bytes < L.total || (reinterpret_cast<uintptr_t>(workspace) % kAl))
        return FBSDE_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const cudaError_t e = launch_call(P, L, K, direct, Q, x0, seed, solve_index0, u0, grad_u0,
                                      static_cast<char *>(workspace), s);
    return e == cudaSuccess ? FBSDE_OK : FBSDE_ERR_CUDA;
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
    return P ? fbsde_solve_batch(P, P->M, Q, x0, seed, solve_index0, u0, grad_u0, workspace,
                                 workspace_bytes, stream)
             : FBSDE_ERR_ARG;
}


int fbsde_solve_batch(const fbsde_problem *P, int64_t K, int32_t Q, const double *x0,
                      uint64_t seed, uint32_t solve_index0, double *u0, double *grad_u0,
                      void *workspace, size_t workspace_bytes, fbsde_stream_t stream)
{
    return solve_batch(P, K, false, Q, x0, seed, solve_index0, u0, grad_u0, workspace,
                       workspace_bytes, stream);
}

int fbsde_solve_batch_direct(const fbsde_problem *P, int64_t K, int32_t Q, const double *x0,
                             uint64_t seed, uint32_t solve_index0, double *u0, double *grad_u0,
                             void *workspace, size_t workspace_bytes, fbsde_stream_t stream)
{
    static_assert(kDirMaxD == FBSDE_BATCH_DIRECT_MAX_D, "the header's limit");
    return solve_batch(P, K, true, Q, x0, seed, solve_index0, u0, grad_u0, workspace,
                       workspace_bytes, stream);
}

int fbsde_anchored_diagnostics(const fbsde_problem *P, const void *workspace, fbsde_diag *out,
                               fbsde_stream_t stream)
{
    Lay L;
    if (!lay(P, L) || !workspace || !out) return FBSDE_ERR_ARG;
    int h[4] = {0, 0, 0, 0};
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(h, static_cast<const char *>(workspace) + L.cnt, sizeof(h),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return FBSDE_ERR_CUDA;
    std::memset(out, 0, sizeof(*out));
    out->status = h[1];
    out->cg_iters_total = h[3];
    return FBSDE_OK;
}

}  // extern "C"
