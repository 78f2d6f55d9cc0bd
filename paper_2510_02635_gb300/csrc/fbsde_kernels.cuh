// fbsde_kernels.cuh -- CUDA kernels of the localized FBSDE scheme, templated on the
// precision Real of the particle stream (float or double).  Included once per
// precision by fbsde_kernels_f32.cu / fbsde_kernels_f64.cu.
//
// Kernel families of one solve (query points s = 0..Q-1 in one launch each):
//   k_forward, k_update    row-segment kernels: one warp per (s, particle, segment),
//                          Philox/Box-Muller in registers, the particle row updated in
//                          place, per-segment partial sums written out (no barriers);
//   k_particles            one thread per particle: segment sums, FP64 Newton, kernel
//                          weights and the three moment coefficients;
//   k_moments              streaming weighted column sums of the particle rows;
//   k_matvec               the matrix-free product of the regression operator (a team
//                          of warps per row: dot product, then the weighted row sum);
//   k_reduce_partials      fixed-order compensated sum of the per-CTA partial vectors,
//                          and in the CG the operator's FP64 epilogue (tiles of 128);
//   k_cg_update            one CG pass of the d-vectors, tiles of 128 elements per block;
//   k_moments_finalize, k_cg_post, k_setup
//                          one CTA per query: FP64 d-vector algebra of the regression.
#pragma once
#include <math.h>

#include "fbsde_internal.cuh"

namespace fbsde {
namespace dev {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64
// products whose halves are xored with the other two words and the round key; the
// key advances by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        // the two 32 x 32 -> 64-bit products, high and low halves from one multiply each
        const unsigned long long p0 = (unsigned long long)c.x * 0xD2511F53u;
        const unsigned long long p1 = (unsigned long long)c.z * 0xCD9E8D57u;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
    }
    return c;
}

// The same generator with the ten round keys precomputed (rk0[r] = k0 + r W0,
// rk1[r] = k1 + r W1), read from the kernel's parameter space.
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const uint32_t *rk0,
                                                  const uint32_t *rk1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const unsigned long long p0 = (unsigned long long)c.x * 0xD2511F53u;
        const unsigned long long p1 = (unsigned long long)c.z * 0xCD9E8D57u;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk0[round], (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ rk1[round], (uint32_t)p0);
    }
    return c;
}

// Hardware approximations of the special-function unit with denormal inputs and results
// flushed to zero (every argument they get here is a normal number: u >= 2^-24, L >= 1e-7,
// angles and coordinates of order one), so no denormal range fix-up is compiled around
// them: base-2 logarithm, reciprocal, reciprocal square root, sine and cosine of an angle
// in radians.
__device__ __forceinline__ float lg2_ftz(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_ftz(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sin_ftz(float x)
{
    float y;
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float cos_ftz(float x)
{
    float y;
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 32-bit word -> ((x >> 9) + 1/2) 2^-23 in (0,1), exact in binary32: the funnel shift puts
// the top 23 bits of x under the exponent bits of 1.0 (0x7F << 23), giving
// 1 + (x >> 9) 2^-23 in [1, 2); subtracting 1 - 2^-24 is exact, since the result
// (2 (x >> 9) + 1) 2^-24 has at most 24 significant bits.
__device__ __forceinline__ float u01f(uint32_t x)
{
    return __uint_as_float(__funnelshift_r(x, 0x7Fu, 9)) - (1.0f - 0x1p-24f);
}
__device__ __forceinline__ double u01d(uint32_t x)
{
    return ((double)(x >> 9) + 0.5) * 0x1p-23;
}

// ln u for u in (0, 1) in FP32.  For u <= 3/4 the hardware base-2 logarithm times ln 2,
// whose error is small relative to |ln u| >= 0.287 there; above, where ln u -> 0 and an
// absolute error would dominate, the series ln u = 2 atanh(s) = 2 (s + s^3/3 + s^5/5 +
// s^7/7 + s^9/9), s = (u - 1)/(u + 1) in [-1/7, 0) (u - 1 is exact; the next term is below
// 2e-9 relative).  Both are evaluated and one selected, so the warp does not diverge.
__device__ __forceinline__ float ln_unit(float u)
{
    const float s = (u - 1.0f) * rcp_ftz(u + 1.0f);
    const float s2 = s * s;
    float p = fmaf(s2, 1.0f / 9.0f, 1.0f / 7.0f);
    p = fmaf(s2, p, 0.2f);
    p = fmaf(s2, p, 1.0f / 3.0f);
    p = fmaf(s2, p, 1.0f);
    const float near1 = 2.0f * s * p;
    return u > 0.75f ? near1 : lg2_ftz(u) * 0.693147180559945309f;
}

// Box-Muller (1958): (a, b) -> sqrt(-2 ln u_a) (cos, sin)(2 pi u_b), times `scale`.
// FP32: ln_unit; sqrt(L) as L / sqrt(L) with the hardware reciprocal square root; the angle
// taken as theta = 2 pi u_b - pi in (-pi, pi), where the hardware sine and cosine are
// accurate to 3.4e-7 absolute (measured on every u_b of the 2^23-point grid), and
// (cos, sin)(2 pi u_b) = -(cos, sin)(theta), the sign folded into the radius.  The normals
// stay within 2e-6 of the FP64 transform of the same words.  The scale (the path
// step's sigma sqrt(dt) factor) multiplies the radius once per pair; scale = 1 gives the
// normals themselves.
__device__ __forceinline__ void box_muller_scaled(uint32_t a, uint32_t b, float scale, float &z0,
                                                  float &z1)
{
    const float L = -2.0f * ln_unit(u01f(a));
    const float nr = -scale * (L * rsqrt_ftz(L));
    const float th = fmaf(u01f(b), 6.28318530717958648f, -3.14159265358979324f);
    z0 = nr * cos_ftz(th);
    z1 = nr * sin_ftz(th);
}
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float &z0, float &z1)
{
    box_muller_scaled(a, b, 1.0f, z0, z1);
}
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, double &z0, double &z1)
{
    const double r = sqrt(-2.0 * log(u01d(a)));
    double sn, cs;
    sincospi(2.0 * u01d(b), &sn, &cs);
    z0 = r * cs;
    z1 = r * sn;
}

// 16 bytes of a particle row: 4 floats or 2 doubles.
template <typename Real> struct alignas(16) Chunk {
    static constexpr int E = 16 / sizeof(Real);
    Real v[E];
};

template <typename Real> __device__ __forceinline__ Chunk<Real> ld_chunk(const Real *p)
{
    Chunk<Real> c;
    *reinterpret_cast<int4 *>(c.v) = *reinterpret_cast<const int4 *>(p);
    return c;
}
template <typename Real> __device__ __forceinline__ Chunk<Real> ldg_chunk(const Real *p)
{
    Chunk<Real> c;
    *reinterpret_cast<int4 *>(c.v) = __ldg(reinterpret_cast<const int4 *>(p));
    return c;
}
template <typename Real> __device__ __forceinline__ void st_chunk(Real *p, const Chunk<Real> &c)
{
    *reinterpret_cast<int4 *>(p) = *reinterpret_cast<const int4 *>(c.v);
}
template <typename Real> __device__ __forceinline__ void zero(Chunk<Real> &c)
{
#pragma unroll
    for (int e = 0; e < Chunk<Real>::E; ++e) c.v[e] = Real(0);
}

// Normals xi_{s,k,j,i} for the elements i of chunk c (counter (i/4, j, k, s)); the
// elements at i >= d are zero.
__device__ __forceinline__ Chunk<float> normal_chunk(Chunk<float> *, int c, uint32_t j, uint32_t k,
                                                     uint32_t s, uint32_t k0, uint32_t k1, int d)
{
    const uint4 w = philox4x32_10(make_uint4((uint32_t)c, j, k, s), k0, k1);
    Chunk<float> z;
    box_muller(w.x, w.y, z.v[0], z.v[1]);
    box_muller(w.z, w.w, z.v[2], z.v[3]);
    const int i0 = 4 * c;
#pragma unroll
    for (int e = 0; e < 4; ++e)
        if (i0 + e >= d) z.v[e] = 0.0f;
    return z;
}
__device__ __forceinline__ Chunk<double> normal_chunk(Chunk<double> *, int c, uint32_t j, uint32_t k,
                                                      uint32_t s, uint32_t k0, uint32_t k1, int d)
{
    const uint4 w = philox4x32_10(make_uint4((uint32_t)(c >> 1), j, k, s), k0, k1);
    Chunk<double> z;
    if (c & 1)
        box_muller(w.z, w.w, z.v[0], z.v[1]);
    else
        box_muller(w.x, w.y, z.v[0], z.v[1]);
    const int i0 = 2 * c;
#pragma unroll
    for (int e = 0; e < 2; ++e)
        if (i0 + e >= d) z.v[e] = 0.0;
    return z;
}

// ---------------------------------------------------------------------------
// Reductions.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void bar_named(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

struct Team {
    int tw, tthreads, team, tl, lane, wt, nteams;
    __device__ __forceinline__ explicit Team(int team_warps)
    {
        tw = team_warps;
        tthreads = 32 * tw;
        team = threadIdx.x / tthreads;
        tl = threadIdx.x - team * tthreads;
        lane = threadIdx.x & 31;
        wt = tl >> 5;
        nteams = blockDim.x / tthreads;
    }
};

// Sum over the threads of one team.  The xor butterfly leaves the same bits in every
// lane (each step adds two lane values that are already equal pairwise, and addition
// commutes); the cross-warp step reads the warp sums in warp order.  slots:
// [nteams][2][32][NV], double-buffered so that one named barrier per call suffices.
template <typename T, int NV>
__device__ __forceinline__ void team_sum(T (&v)[NV], T *slots, const Team &tm, int &phase)
{
#pragma unroll
    for (int i = 0; i < NV; ++i) {
#pragma unroll
        for (int o = 16; o; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    }
    if (tm.tw == 1) return;
    T *sl = slots + (size_t)((tm.team * 2 + phase) * 32) * NV;
    if (tm.lane == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) sl[tm.wt * NV + i] = v[i];
    }
    bar_named(1 + tm.team, tm.tthreads);
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        T a = T(0);
        for (int w = 0; w < tm.tw; ++w) a += sl[w * NV + i];
        v[i] = a;
    }
    phase ^= 1;
}

// Block-wide sum of NV doubles (all threads receive the same bits).  sm: [32][NV].
template <int NV> __device__ __forceinline__ void block_sum(double (&v)[NV], double *sm)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
#pragma unroll
        for (int o = 16; o; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    }
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) sm[warp * NV + i] = v[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        double a = 0.0;
        for (int w = 0; w < nw; ++w) a += sm[w * NV + i];
        v[i] = a;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Problem table (the same formulas as documented in fbsde.h).
// ---------------------------------------------------------------------------
// cos of a particle coordinate in the stream precision.  FP32: x - 2 pi n with
// n = rint(x / (2 pi)) by a two-part 2 pi (Cody and Waite 1980: 6.28125 has 8 significant
// bits, so n * 6.28125 is exact for |n| < 2^16), then the hardware cosine on [-pi, pi]
// (absolute error below 1e-6).  The coordinates enter only through sums over d terms of
// FP32 values (the Allen-Cahn feature sum_i cos x_i), so this is within the stream's
// rounding; it replaces the range reduction and polynomial of the accurate cosf, which
// dominate the instruction count of the row kernels.  FP64: cos.
__device__ __forceinline__ float cos_stream(float x)
{
    const float n = rintf(x * 0.15915494309189535f);
    float r = fmaf(-n, 6.28125f, x);
    r = fmaf(-n, 1.9353071795864769e-3f, r);
    return __cosf(r);
}
__device__ __forceinline__ double cos_stream(double x) { return cos(x); }
// sin with the same reduction (the drift kinds' source terms).
__device__ __forceinline__ float sin_stream(float x)
{
    const float n = rintf(x * 0.15915494309189535f);
    float r = fmaf(-n, 6.28125f, x);
    r = fmaf(-n, 1.9353071795864769e-3f, r);
    return __sinf(r);
}
__device__ __forceinline__ double sin_stream(double x) { return sin(x); }

// Per-element term of the terminal feature sum; x = x0_i + Delta_i.
template <typename Real> __device__ __forceinline__ Real g_term(int kind, Real x, Real th)
{
    switch (kind) {
    case FBSDE_AC_MANUFACTURED:
    case FBSDE_COS_LINEAR_TEST: return cos_stream(x);
    case FBSDE_LOGISTIC_GRAD: return x;
    case FBSDE_HJB_LOGQUAD: return th * x * x;
    case FBSDE_AFFINE_TEST: return th * x;
    case FBSDE_AC_DOUBLEWELL: return x * x;
    default: return Real(0);
    }
}

// g from its feature sum phi.
__device__ __forceinline__ double g_value(const Params &p, double phi)
{
    switch (p.kind) {
    case FBSDE_AC_MANUFACTURED:
    case FBSDE_COS_LINEAR_TEST: return phi / p.d;
    case FBSDE_LOGISTIC_GRAD: return 1.0 / (1.0 + exp(-(p.T + phi / p.d)));
    case FBSDE_HJB_LOGQUAD: return log(0.5 * (1.0 + phi));
    case FBSDE_AFFINE_TEST: return p.A + phi;
    case FBSDE_CUBIC_TEST: return p.A;
    case FBSDE_AC_DOUBLEWELL: return 1.0 / (2.0 + 0.4 * phi);
    case FBSDE_DRIFT_AC:
    case FBSDE_DRIFT_QUAD: return phi / p.d;
    }
    return NAN;
}

// The y-independent part of f at time t: AC_MANUFACTURED uses phi = sum_i cos x_i,
// the z-dependent kinds use sum_i z_i and |z|^2 of the level, the drift kinds the sums
// phi (of g's terms) and psi of their source:
//   DRIFT_AC:   u*^3 - 2 u* + e^{t-T} psi / d,  psi = sum_i s_i^2 cos x_i / 2 + m_i sin x_i;
//   DRIFT_QUAD: u*^3 - 2 u* - e^{t-T} psi / d,  psi = sum_i s_i^2 + 2 m_i x_i;
// u* = e^{t-T} phi / d, s_i = sigma + sig1 x_i, m_i = mu0 + mu1 x_i (these sources make u*
// the exact solution of (2.1) under the drift mu and the diffusion diag(s)).
__device__ __forceinline__ double f_feature(const Params &p, double t, double phi, double sumz,
                                            double zz, double psi = 0.0)
{
    switch (p.kind) {
    case FBSDE_AC_MANUFACTURED: {
        const double us = exp(t - p.T) * phi / p.d;
        return us * us * us - (2.0 - 0.5 * p.sigma * p.sigma) * us;
    }
    case FBSDE_DRIFT_AC:
    case FBSDE_DRIFT_QUAD: {
        const double e = exp(t - p.T), us = e * phi / p.d;
        const double q = e * psi / p.d;
        return us * us * us - 2.0 * us + (p.kind == FBSDE_DRIFT_AC ? q : -q);
    }
    case FBSDE_LOGISTIC_GRAD: return sumz;
    case FBSDE_HJB_LOGQUAD: return zz;
    case FBSDE_AFFINE_TEST: return p.c2 * sumz + p.c3 * t;
    }
    return 0.0;
}

__device__ __forceinline__ double f_scalar(const Params &p, double feat, double y, double &dfdy)
{
    switch (p.kind) {
    case FBSDE_AC_MANUFACTURED:
    case FBSDE_DRIFT_AC:
    case FBSDE_DRIFT_QUAD:
        dfdy = 1.0 - 3.0 * y * y;
        return y - y * y * y + feat;
    case FBSDE_LOGISTIC_GRAD:
        dfdy = feat;
        return (y - (2.0 + p.d) / (2.0 * p.d)) * feat;
    case FBSDE_HJB_LOGQUAD:
        dfdy = 0.0;
        return -0.5 * feat;
    case FBSDE_AFFINE_TEST:
        dfdy = p.c1;
        return p.c0 + p.c1 * y + feat;
    case FBSDE_COS_LINEAR_TEST:
        dfdy = p.c1;
        return p.c0 + p.c1 * y;
    case FBSDE_CUBIC_TEST:
    case FBSDE_AC_DOUBLEWELL:
        dfdy = 1.0 - 3.0 * y * y;
        return y - y * y * y;
    }
    dfdy = NAN;
    return NAN;
}

// Newton iteration (2.17) on F(Y) = Y - E_hat - dt f (2.16), from Y = E_hat.
// iters = iterations used, or -1 if newton_max_iter ran out.
__device__ __forceinline__ double newton(const Params &p, double E_hat, double feat, int &iters)
{
    double y = E_hat;
    for (int n = 1; n <= p.newton_max_iter; ++n) {
        double dfdy;
        const double f = f_scalar(p, feat, y, dfdy);
        const double F = y - E_hat - p.dt * f;
        const double dF = 1.0 - p.dt * dfdy;
        const double dy = F / dF;
        y -= dy;
        if (fabs(dy) <= p.newton_tol * fmax(1.0, fabs(y))) {
            iters = n;
            return y;
        }
    }
    iters = -1;
    return y;
}

// Unnormalised Gaussian kernel weight exp(-(rho - rho_ref) / (h^2 rho_ref)) (Remark 2.3);
// the shift by rho_ref = E|D|^2 cancels in the normalisation.
__device__ __forceinline__ double kernel_weight(const Params &p, double rho, double rho_ref)
{
    return p.uniform ? 1.0 : exp(-(rho - rho_ref) / (p.h2 * rho_ref));
}


// ---------------------------------------------------------------------------
// Workspace accessors.
// ---------------------------------------------------------------------------
template <typename Real> struct WS {
    const Params &p;
    __device__ __forceinline__ explicit WS(const Params &pp) : p(pp) {}
    __device__ __forceinline__ Real *row(int s, long long j) const
    {
        return reinterpret_cast<Real *>(p.delta) + ((size_t)s * p.M + j) * p.ld;
    }
    __device__ __forceinline__ Real *w(int s) const
    {
        return reinterpret_cast<Real *>(p.w) + (size_t)s * p.M;
    }
    __device__ __forceinline__ double *Y(int s) const { return p.Y + (size_t)s * p.M; }
    // per-particle moment coefficients (w, w (Y - yref), w (D . g)), g the starting guess
    // of the solve
    __device__ __forceinline__ Real *coef(int s, long long j) const
    {
        return reinterpret_cast<Real *>(p.coef) + ((size_t)s * p.M + j) * 3;
    }
    // per-particle, per-row-segment partial sums [kSegSums]
    __device__ __forceinline__ Real *segp(int s, long long j, int seg) const
    {
        return reinterpret_cast<Real *>(p.segp) + (((size_t)s * p.M + j) * p.nseg + seg) * kSegSums;
    }
    __device__ __forceinline__ Real *part(int s, int g, int v) const
    {
        return reinterpret_cast<Real *>(p.part) + (((size_t)s * p.G + g) * kPartVecs + v) * p.ld;
    }
    __device__ __forceinline__ double *spart(int s, int b) const
    {
        return p.spart + ((size_t)s * p.GS + b) * kPartScal;
    }
    // FP64 vectors: 0 x (= alpha_x; after the level, the next level's starting guess),
    // 1 r, 2 p, 3 S, 4 b / rhs, 5 w = A r or G, 6 x0, 7 s = A p, 8 alpha_x of the level
    // before
    __device__ __forceinline__ double *v64(int s, int which) const
    {
        return p.vec64 + ((size_t)s * kVec64 + which) * p.ld;
    }
    // stream-precision vectors: 0 operand of the product (r), 1 alpha_x, 2 x0, 3 the next
    // level's starting guess; theta after all solves
    __device__ __forceinline__ Real *vR(int s, int which) const
    {
        return reinterpret_cast<Real *>(p.vecR) + ((size_t)s * kVecR + which) * p.ld;
    }
    __device__ __forceinline__ Real *thetaR() const
    {
        return reinterpret_cast<Real *>(p.vecR) + (size_t)p.Q * kVecR * p.ld;
    }
    // forward SDE: offset c_k = a_k - x0 of the anchor of the level-k regression
    __device__ __forceinline__ Real *anchor(int s, int k) const
    {
        return reinterpret_cast<Real *>(p.anchor) + ((size_t)s * (p.N + 1) + k) * p.ld;
    }
};

__device__ __forceinline__ void row_range(long long M, int G, int g, long long &r0, long long &r1)
{
    r0 = (long long)((unsigned long long)M * (unsigned long long)g / (unsigned long long)G);
    r1 = (long long)((unsigned long long)M * (unsigned long long)(g + 1) / (unsigned long long)G);
}

template <typename T, int NV> __device__ __forceinline__ void warp_sum(T (&v)[NV])
{
#pragma unroll
    for (int i = 0; i < NV; ++i) {
#pragma unroll
        for (int o = 16; o; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    }
}

// ---------------------------------------------------------------------------
// Row-segment kernels.  Work item = (query s, particle j, segment); one warp per item,
// lane l holding chunks c0 + l + 32 v (v < VPT) of the segment.  Each item writes its
// warp sums to segp; the per-particle kernel adds the segments in order.  No barriers,
// no shared memory, coalesced 512-byte accesses per warp instruction.
// ---------------------------------------------------------------------------

// Grid-stride walk over the items of the row kernels, one warp per item
// it = (s M + j) nseg + seg (query s, particle j, row segment seg): the first item and the
// stride are split into (s, j, seg) once, and each step adds the stride's triple with
// carries, so the loop has no integer division (64-bit division is a long instruction
// sequence, paid per warp item).  M < 2^31 keeps j + dj + carry below 2^32.
struct RowItems {
    uint32_t seg, j, s, dseg, dj, ds, nseg, M;
    __device__ __forceinline__ RowItems(const Params &p, unsigned long long first,
                                        unsigned long long stride)
        : nseg((uint32_t)p.nseg), M((uint32_t)p.M)
    {
        const unsigned long long row = first / nseg, drow = stride / nseg;
        seg = (uint32_t)(first - row * nseg);
        s = (uint32_t)(row / M);
        j = (uint32_t)(row - (unsigned long long)s * M);
        dseg = (uint32_t)(stride - drow * nseg);
        ds = (uint32_t)(drow / M);
        dj = (uint32_t)(drow - (unsigned long long)ds * M);
    }
    __device__ __forceinline__ void next()
    {
        seg += dseg;
        const uint32_t c = seg >= nseg ? 1u : 0u;
        seg -= c * nseg;
        j += dj + c;
        const uint32_t c2 = j >= M ? 1u : 0u;
        j -= c2 * M;
        s += ds + c2;
    }
};

// Forward sweep (2.7) with mu = 0: the increments telescope to Delta_N^j = sigma W^j(T),
// and the Brownian path is drawn backwards from its end point (Brownian bridge, see
// k_update), so Delta_N^j = sigma sqrt(T) xi_{s,N,j} (wb = sigma sqrt(T)), stored;
// segment sums of (|Delta|^2, terminal feature of g at x0 + Delta).
template <typename Real, int VPT>
__global__ void __launch_bounds__(256) k_forward(Params p)
{
    constexpr int E = Chunk<Real>::E;
    const WS<Real> ws(p);
    const int lane = threadIdx.x & 31;
    const int nch = p.ld / E;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const Real wb = (Real)p.wb;
    const bool need_theta = p.kind == FBSDE_HJB_LOGQUAD || p.kind == FBSDE_AFFINE_TEST;
    const Real *thr = ws.thetaR();
    for (RowItems w(p, (((unsigned long long)blockIdx.x * blockDim.x) + threadIdx.x) >> 5,
                    (unsigned long long)nwarps);
         w.s < (uint32_t)p.Q; w.next()) {
        const int seg = (int)w.seg, s = (int)w.s;
        const long long j = w.j;
        const uint32_t sidx = p.solve0 + (uint32_t)s;
        const Real *x0r = ws.vR(s, 2);
        Real *drow = ws.row(s, j);
        Real acc[2] = {Real(0), Real(0)};  // |D|^2, g feature
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            const int c = seg * 32 * VPT + lane + 32 * v;
            if (c < nch) {
                Chunk<Real> dl = normal_chunk((Chunk<Real> *)nullptr, c, (uint32_t)j,
                                              (uint32_t)p.N, sidx, p.key0, p.key1, p.d);
#pragma unroll
                for (int e = 0; e < E; ++e) dl.v[e] *= wb;
                const Chunk<Real> xc = ldg_chunk(x0r + c * E);
                Chunk<Real> th;
                if (need_theta) th = ldg_chunk(thr + c * E);
                else zero(th);
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    acc[0] += dl.v[e] * dl.v[e];
                    if (c * E + e < p.d) acc[1] += g_term(p.kind, xc.v[e] + dl.v[e], th.v[e]);
                }
                st_chunk(drow + c * E, dl);
            }
        }
        warp_sum(acc);
        if (lane == 0) {
            Real *o = ws.segp(s, j, seg);
            o[0] = acc[0];
            o[1] = acc[1];
            o[2] = Real(0);
            o[3] = Real(0);
        }
    }
}

// Level update (1 <= k < N): one step of the Brownian path drawn backwards by the bridge,
// Delta_k = a Delta_{k+1} + b xi_{s,k,j} in place (wa = a = k/(k+1), wb = b =
// sigma sqrt(dt k/(k+1)); the reverse sweep of the adjoint runs the same step solved for
// Delta_{k+1}); segment sums of (alpha_x . Delta_k, |Delta_k|^2, sum_i cos(x0_i + Delta_k,i)
// for the Allen-Cahn source).
template <typename Real, int VPT>
__global__ void __launch_bounds__(256) k_update(Params p)
{
    constexpr int E = Chunk<Real>::E;
    const WS<Real> ws(p);
    const int lane = threadIdx.x & 31;
    const int nch = p.ld / E;
    const int k = p.level;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const Real wa = (Real)p.wa, wb = (Real)p.wb;
    const bool cos_feature = p.kind == FBSDE_AC_MANUFACTURED;
    for (RowItems w(p, (((unsigned long long)blockIdx.x * blockDim.x) + threadIdx.x) >> 5,
                    (unsigned long long)nwarps);
         w.s < (uint32_t)p.Q; w.next()) {
        const int seg = (int)w.seg, s = (int)w.s;
        const long long j = w.j;
        const uint32_t sidx = p.solve0 + (uint32_t)s;
        const Real *xr = ws.vR(s, 1);
        const Real *x0r = ws.vR(s, 2);
        const Real *gr = ws.vR(s, 3);
        Real *drow = ws.row(s, j);
        Chunk<Real> dl[VPT];
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            const int c = seg * 32 * VPT + lane + 32 * v;
            if (c < nch) dl[v] = ld_chunk(drow + c * E);
        }
        Real acc[4] = {Real(0), Real(0), Real(0), Real(0)};
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            const int c = seg * 32 * VPT + lane + 32 * v;
            if (c < nch) {
                const Chunk<Real> z = normal_chunk((Chunk<Real> *)nullptr, c, (uint32_t)j,
                                                   (uint32_t)k, sidx, p.key0, p.key1, p.d);
                const Chunk<Real> xc = ldg_chunk(xr + c * E);
                const Chunk<Real> gc = ldg_chunk(gr + c * E);
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    dl[v].v[e] = wa * dl[v].v[e] + wb * z.v[e];
                    acc[0] += xc.v[e] * dl[v].v[e];
                    acc[1] += dl[v].v[e] * dl[v].v[e];
                    acc[3] += gc.v[e] * dl[v].v[e];
                }
                if (cos_feature) {
                    const Chunk<Real> x0c = ldg_chunk(x0r + c * E);
#pragma unroll
                    for (int e = 0; e < E; ++e)
                        if (c * E + e < p.d) acc[2] += cos_stream(x0c.v[e] + dl[v].v[e]);
                }
                st_chunk(drow + c * E, dl[v]);
            }
        }
        warp_sum(acc);
        if (lane == 0) {
            Real *o = ws.segp(s, j, seg);
            o[0] = acc[0];
            o[1] = acc[1];
            o[2] = acc[2];
            o[3] = acc[3];
        }
    }
}

// ---------------------------------------------------------------------------
// Per-particle scalar work, one thread per particle (grid (ceil(M/256), Q)), FP64.
//   terminal (level = N): Y_N = g(x0 + Delta_N) (Algorithm 1), w = K(|Delta_N|),
//                         coefficients (w, w (Y - g(x0)), 0);
//   level k >= 1:         E_hat = alpha + alpha_x . Delta_k (local affine model), Newton
//                         (2.16)-(2.17) for Y_k, w = K(|Delta_k|) for the level k-1
//                         regression, coefficients (w, w (Y - alpha), w g . Delta_k), g the
//                         starting guess of that regression's solve (k_cg_post).
// Block sums of (w, w (Y - yref), w |D|^2) go to spart in thread order.
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void __launch_bounds__(256) k_particles(Params p)
{
    __shared__ double sm[32 * 4];
    const int s = blockIdx.y;
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const WS<Real> ws(p);
    SolveState &st = p.st[s];
    const bool terminal = p.level == p.N;
    const double t_k = p.level * p.dt;
    // kernel scale: E|Delta_k|^2 = sigma^2 d t_k without a drift; the cloud's mean squared
    // distance to the anchor (k_sde_rho) with one
    const double rho_ref = p.sde ? st.rho_ref : p.sigma * p.sigma * p.d * t_k;
    const double yref = terminal ? st.gx0 : st.alpha;
    double sums[3] = {0.0, 0.0, 0.0};
    int it_used = 0, failed = 0;
    if (j < p.M) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0, a4 = 0.0, a5 = 0.0;
        for (int seg = 0; seg < p.nseg; ++seg) {
            const Real *sp = ws.segp(s, j, seg);
            a0 += (double)sp[0];
            a1 += (double)sp[1];
            a2 += (double)sp[2];
            a3 += (double)sp[3];
            if (p.sde) {
                a4 += (double)sp[4];
                a5 += (double)sp[5];
            }
        }
        double Yj, rho, dot = 0.0;
        if (p.sde) {
            // rows of k_sde_rows: [0] alpha_x . Delta, [1] |Delta|^2, [2] |Delta - c_{k-1}|^2,
            // [3] g . Delta, [4], [5] feature sums.  Level k < N: the prediction at the drifted
            // position, alpha + alpha_x . (Delta + mu(x0 + Delta) dt) with alpha the intercept
            // at Delta = 0, and Z = sigma(X)^T alpha_x, so sum_i z_i = sigma sum alpha_x +
            // sig1 alpha_x . (x0 + Delta) and |z|^2 = sigma^2 |alpha_x|^2 (sig1 = 0 there).
            if (terminal) {
                Yj = g_value(p, a4);
            } else {
                const double E_hat = st.alpha + (1.0 + p.mu1 * p.dt) * a0 +
                                     p.dt * (p.mu0 * st.sum_ax + p.mu1 * st.ax_x0);
                const double sumz = st.sumz + p.sig1 * (st.ax_x0 + a0);
                const double feat = p.kind == FBSDE_AC_MANUFACTURED
                                        ? f_feature(p, t_k, a4, 0.0, 0.0)
                                        : f_feature(p, t_k, a4, sumz, st.zz, a5);
                int it;
                Yj = newton(p, E_hat, feat, it);
                if (it < 0) {
                    failed = 1;
                    it_used = p.newton_max_iter;
                } else {
                    it_used = it;
                }
            }
            rho = a2;   // distance to the anchor: the kernel weight
            a2 = a1;    // |Delta|^2: the trace of the weighted covariance (shift-free)
        } else if (terminal) {
            rho = a0;
            Yj = g_value(p, a1);
            a2 = rho;
        } else {
            dot = a0;
            rho = a1;
            const double feat = p.kind == FBSDE_AC_MANUFACTURED
                                    ? f_feature(p, t_k, a2, 0.0, 0.0)
                                    : f_feature(p, t_k, 0.0, st.sumz, st.zz);
            int it;
            Yj = newton(p, st.alpha + dot, feat, it);
            if (it < 0) {
                failed = 1;
                it_used = p.newton_max_iter;
            } else {
                it_used = it;
            }
            a2 = rho;
        }
        const Real wr = (Real)kernel_weight(p, rho, rho_ref);
        const double wd = (double)wr;
        ws.Y(s)[j] = Yj;
        ws.w(s)[j] = wr;
        if (p.tape_w) {  // record Y_level and the weights of regression level-1
            p.tape_Y[((size_t)p.level * p.Q + s) * p.M + j] = Yj;
            reinterpret_cast<Real *>(p.tape_w)[((size_t)(p.level - 1) * p.Q + s) * p.M + j] = wr;
        }
        Real *cf = ws.coef(s, j);
        cf[0] = wr;
        cf[1] = (Real)(wd * (Yj - yref));
        cf[2] = (Real)(wd * a3);   // D . (starting guess of the next level's solve)
        sums[0] = wd;
        sums[1] = wd * (Yj - yref);
        sums[2] = wd * a2;
    }
    block_sum(sums, sm);
    if (threadIdx.x == 0) {
        double *o = ws.spart(s, blockIdx.x);
        o[0] = sums[0];
        o[1] = sums[1];
        o[2] = sums[2];
    }
    if (!terminal) {
        int mx = it_used;
#pragma unroll
        for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        const bool any_failed = __any_sync(0xffffffffu, failed);
        if ((threadIdx.x & 31) == 0) {
            if (mx) {
                atomicMax(&st.newton_max, mx);
                atomicMax(&st.newton_max_all, mx);
            }
            if (any_failed) atomicCAS(&st.status, 0, (int)FBSDE_ERR_NEWTON);
        }
    }
}

// ---------------------------------------------------------------------------
// Weighted moments of the next regression, a streaming column sum with three weights
// per row: partial_g = (sum w D, sum w (Y - yref) D, sum w (D . g) D) over the rows
// of CTA g.  Grid (tiles, G, Q); a tile covers 256 VM chunks of the row; threads form
// R row groups of tpr threads (R > 1 only for narrow rows), summed in group order.
// ---------------------------------------------------------------------------
template <typename Real, int VM>
__global__ void __launch_bounds__(256) k_moments(Params p)
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
        // rows in order; the loads of kU rows are issued before their sums so that
        // several row chunks are in flight per thread
        constexpr int kU = 4;
        long long j = r0 + rg;
        for (; j + (kU - 1) * R < r1; j += kU * R) {
            Chunk<Real> dl[kU][VM];
            Real cw[kU][3];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const Real *cf = ws.coef(s, j + u * R);
                cw[u][0] = cf[0];
                cw[u][1] = cf[1];
                cw[u][2] = cf[2];
                const Real *drow = ws.row(s, j + u * R);
#pragma unroll
                for (int v = 0; v < VM; ++v) {
                    const int c = c0 + tc + tpr * v;
                    if (c - c0 < tile_nch) dl[u][v] = ld_chunk(drow + c * E);
                }
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
#pragma unroll
                for (int v = 0; v < VM; ++v) {
                    const int c = c0 + tc + tpr * v;
                    if (c - c0 < tile_nch) {
#pragma unroll
                        for (int e = 0; e < E; ++e) {
                            acc[0][v].v[e] += cw[u][0] * dl[u][v].v[e];
                            acc[1][v].v[e] += cw[u][1] * dl[u][v].v[e];
                            acc[2][v].v[e] += cw[u][2] * dl[u][v].v[e];
                        }
                    }
                }
            }
        }
        for (; j < r1; j += R) {
            const Real *cf = ws.coef(s, j);
            const Real w0 = cf[0], w1 = cf[1], w2 = cf[2];
            const Real *drow = ws.row(s, j);
#pragma unroll
            for (int v = 0; v < VM; ++v) {
                const int c = c0 + tc + tpr * v;
                if (c - c0 < tile_nch) {
                    const Chunk<Real> dl = ld_chunk(drow + c * E);
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        acc[0][v].v[e] += w0 * dl.v[e];
                        acc[1][v].v[e] += w1 * dl.v[e];
                        acc[2][v].v[e] += w2 * dl.v[e];
                    }
                }
            }
        }
    }
    if (R == 1) {
        if (rg >= R) return;  // threads beyond one row group own no chunk
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
    // narrow rows: reduce the R row groups through shared memory, in group order
    Real *red = reinterpret_cast<Real *>(smem_raw);  // [R][3][tile_nch][E]
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

// Sum of the G per-CTA partial vectors in a fixed order.  Block = 32 lanes x GR groups
// (GR = blockDim.x / 32 >= 4) over a tile of kRedTile = 128 elements; lane l owns the four
// consecutive elements 4l..4l+3 of the tile.  Group gg adds partials g = gg, gg + GR, ...
// in order (loads issued eight at a time), then thread t < 128 adds the GR group sums of
// element t in group order.  With FP32 partials every addition is compensated (Neumaier
// 1974): the running sum and its error term stay in FP32 and only the final s + c is
// widened to FP64.  FP64 partials are added in FP64.
//   cg_mode = 0: vectors 0..nvec-1 into v64 slots dst0..
//   cg_mode = 1: the product of the CG pass (queries already converged skip):
//       w = sum / W - S (S . r) + lambda r   (Gamma_c r + lambda r, Eq. 3.19's operator)
//     into slot 5 and this block's share of w . r into bpart; every block of k_cg_update
//     adds the shares and derives the pass's scalars from them.
// Grid (nblk, Q), nblk = ceil(ld / kRedTile).
template <typename Real> struct RedAcc {
    double s;
    __device__ __forceinline__ void init() { s = 0.0; }
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ void merge(double x, double) { s += x; }
    __device__ __forceinline__ double hi() const { return s; }
    __device__ __forceinline__ double lo() const { return 0.0; }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct RedAcc<float> {
    float s, c;
    __device__ __forceinline__ void init() { s = 0.0f; c = 0.0f; }
    __device__ __forceinline__ void add(float x)
    {
        const float t = __fadd_rn(s, x);
        c = __fadd_rn(c, fabsf(s) >= fabsf(x) ? __fadd_rn(__fsub_rn(s, t), x)
                                               : __fadd_rn(__fsub_rn(x, t), s));
        s = t;
    }
    __device__ __forceinline__ void merge(float xs, float xc)
    {
        add(xs);
        c = __fadd_rn(c, xc);
    }
    __device__ __forceinline__ float hi() const { return s; }
    __device__ __forceinline__ float lo() const { return c; }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

template <typename Real> struct Quad {
    Real v[4];
};
template <typename Real> __device__ __forceinline__ Quad<Real> ld_quad(const Real *p)
{
    Quad<Real> q;
    if constexpr (sizeof(Real) == 4) {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        q.v[0] = t.x; q.v[1] = t.y; q.v[2] = t.z; q.v[3] = t.w;
    } else {
        const double2 a = *reinterpret_cast<const double2 *>(p);
        const double2 b = *reinterpret_cast<const double2 *>(p + 2);
        q.v[0] = a.x; q.v[1] = a.y; q.v[2] = b.x; q.v[3] = b.y;
    }
    return q;
}

template <typename Real>
__global__ void __launch_bounds__(512) k_reduce_partials(Params p, int nvec, int dst0, int cg_mode)
{
    using Acc = RedAcc<Real>;
    using Lo = decltype(Acc{}.lo());
    constexpr int kB = 8;  // loads in flight per lane
    __shared__ Real sh_s[16][kRedTile];
    __shared__ Lo sh_c[16][kRedTile];
    __shared__ double sh_w[4];
    const int s = blockIdx.y;
    SolveState &st = p.st[s];
    if (cg_mode && st.done) return;
    const int lane = threadIdx.x & 31, gg = threadIdx.x >> 5, GR = blockDim.x >> 5;
    const int e0 = blockIdx.x * kRedTile + 4 * lane;  // first element of this lane
    const bool in = e0 < p.ld;                        // ld is a multiple of 4
    const WS<Real> ws(p);
    const size_t stride = (size_t)kPartVecs * p.ld * GR;   // between this group's partials
    for (int v = 0; v < nvec; ++v) {
        Acc acc[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[e].init();
        if (in) {
            const Real *src = ws.part(s, gg, v) + e0;
            for (int g0 = gg; g0 < p.G; g0 += kB * GR, src += kB * stride) {
                Quad<Real> t[kB];
#pragma unroll
                for (int u = 0; u < kB; ++u)
                    if (g0 + u * GR < p.G) t[u] = ld_quad(src + u * stride);
#pragma unroll
                for (int u = 0; u < kB; ++u) {
                    if (g0 + u * GR < p.G) {
#pragma unroll
                        for (int e = 0; e < 4; ++e) acc[e].add(t[u].v[e]);
                    }
                }
            }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            sh_s[gg][4 * lane + e] = acc[e].hi();
            sh_c[gg][4 * lane + e] = acc[e].lo();
        }
        __syncthreads();
        if (threadIdx.x < kRedTile) {
            const int t = threadIdx.x, i = blockIdx.x * kRedTile + t;
            Acc tot;
            tot.init();
            for (int k = 0; k < GR; ++k) tot.merge(sh_s[k][t], sh_c[k][t]);
            const double sum = tot.value();
            if (!cg_mode) {
                if (i < p.ld) ws.v64(s, dst0 + v)[i] = sum;
            } else {
                double wr = 0.0;
                if (i < p.ld) {
                    const double ri = ws.v64(s, 1)[i];
                    const double wi = sum * st.invW - ws.v64(s, 3)[i] * st.sp + st.lambda * ri;
                    ws.v64(s, 5)[i] = wi;
                    wr = wi * ri;
                }
#pragma unroll
                for (int o = 16; o; o >>= 1) wr += __shfl_xor_sync(0xffffffffu, wr, o);
                if (lane == 0) sh_w[t >> 5] = wr;
            }
        }
        __syncthreads();
    }
    if (!cg_mode) return;
    if (threadIdx.x == 0)   // the next kernel boundary makes the shares visible
        p.bpart[((size_t)s * p.nblk + blockIdx.x) * kBpart] = ((sh_w[0] + sh_w[1]) + sh_w[2]) + sh_w[3];
}

// ---------------------------------------------------------------------------
// One CTA per query: set-up of the query point.
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void __launch_bounds__(kFinThreads) k_setup(Params p, const double *x0, const double *theta)
{
    __shared__ double sm[32 * 4];
    const int s = blockIdx.x;
    const WS<Real> ws(p);
    double *x = ws.v64(s, 0), *x0v = ws.v64(s, 6);
    Real *pR = ws.vR(s, 0), *xR = ws.vR(s, 1), *x0R = ws.vR(s, 2);
    // sum cos, sum x, sum x^2, theta-weighted sum, the two drift kinds' psi at x0
    double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    #pragma unroll 4
    for (int i = threadIdx.x; i < p.ld; i += blockDim.x) {
        const double xi = i < p.d ? x0[(size_t)s * p.d + i] : 0.0;
        const double th = (theta && i < p.d) ? theta[i] : 0.0;
        x0v[i] = xi;
        x0R[i] = (Real)xi;
        x[i] = 0.0;
        xR[i] = Real(0);
        pR[i] = Real(0);
        ws.vR(s, 3)[i] = Real(0);
        for (int v = 1; v < kVec64; ++v)
            if (v != 6) ws.v64(s, v)[i] = 0.0;
        if (s == 0) ws.thetaR()[i] = (Real)th;
        if (i < p.d) {
            acc[0] += cos(xi);
            acc[1] += xi;
            acc[2] += xi * xi;
            acc[3] += p.kind == FBSDE_HJB_LOGQUAD ? th * xi * xi : th * xi;
            if (p.sde) {
                const double sg = p.sigma + p.sig1 * xi, m = p.mu0 + p.mu1 * xi;
                acc[4] += 0.5 * sg * sg * cos(xi) + m * sin(xi);
                acc[5] += sg * sg + 2.0 * m * xi;
            }
        }
    }
    block_sum(acc, sm);
    if (threadIdx.x == 0) {
        SolveState st = {};
        double phi = 0.0;
        switch (p.kind) {
        case FBSDE_AC_MANUFACTURED:
        case FBSDE_COS_LINEAR_TEST: phi = acc[0]; break;
        case FBSDE_LOGISTIC_GRAD: phi = acc[1]; break;
        case FBSDE_HJB_LOGQUAD:
        case FBSDE_AFFINE_TEST: phi = acc[3]; break;
        case FBSDE_AC_DOUBLEWELL: phi = acc[2]; break;
        case FBSDE_DRIFT_AC: phi = acc[0]; st.psi0 = acc[4]; break;
        case FBSDE_DRIFT_QUAD: phi = acc[2]; st.psi0 = acc[5]; break;
        }
        // phi0: the feature sum of f at x0 (sum cos x0 of the Allen-Cahn source; phi of g for
        // the drift kinds)
        st.phi0 = p.kind == FBSDE_DRIFT_QUAD ? acc[2] : acc[0];
        st.gx0 = g_value(p, phi);
        st.yref = st.gx0;
        p.st[s] = st;
    }
}

// ---------------------------------------------------------------------------
// One CTA per query: the level-k regression from the reduced moments.
//   S = sum w D / W, b' = sum w (Y - yref) D / W, c' = sum w (Y - yref) / W,
//   lambda = ridge_rel (sum w |D|^2 / W - |S|^2) / d            (ridge of Remark 2.2)
//   rhs = b' - c' S                                              (right side of Eq. 3.19)
//   Gamma_c x = sum w (D . x) D / W - S (S . x)  (x = previous level's alpha_x, or 0)
//   r = p = rhs - Gamma_c x - lambda x,  c = c' + yref.
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void __launch_bounds__(kFinThreads) k_moments_finalize(Params p, int warm)
{
    __shared__ double sm[32 * 4];
    const int s = blockIdx.x;
    const WS<Real> ws(p);
    SolveState &st = p.st[s];
    // per-block scalar sums (W, sum w (Y - yref), sum w |D|^2): strided over the threads,
    // then the block tree (fixed order; a serial FP64 chain over hundreds of blocks would
    // cost 64 cycles per dependent add)
    double ws3[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < p.nsp; b += blockDim.x) {
        const double *sp = ws.spart(s, b);
        ws3[0] += sp[0];
        ws3[1] += sp[1];
        ws3[2] += sp[2];
    }
    block_sum(ws3, sm);
    const double W = ws3[0], Cp = ws3[1], Rr = ws3[2];
    const double invW = 1.0 / W, cp = Cp * invW;
    double *x = ws.v64(s, 0), *r = ws.v64(s, 1), *pp = ws.v64(s, 2), *S = ws.v64(s, 3),
           *B = ws.v64(s, 4), *Gx = ws.v64(s, 5);
    Real *pR = ws.vR(s, 0);
    double a1[2] = {0.0, 0.0};  // |S|^2, S.x
    #pragma unroll 4
    for (int i = threadIdx.x; i < p.ld; i += blockDim.x) {
        S[i] *= invW;
        B[i] *= invW;
        Gx[i] *= invW;
        if (!warm) x[i] = 0.0;
        a1[0] += S[i] * S[i];
        a1[1] += S[i] * x[i];
    }
    block_sum(a1, sm);
    const double lambda = p.ridge_rel * (Rr * invW - a1[0]) / p.d;
    const double sx = a1[1];
    double a2[3] = {0.0, 0.0, 0.0};  // |rhs|^2, |r|^2, S.r
    #pragma unroll 4
    for (int i = threadIdx.x; i < p.ld; i += blockDim.x) {
        const double rhs = B[i] - cp * S[i];
        const double ri = rhs - (Gx[i] - S[i] * sx) - lambda * x[i];
        B[i] = rhs;
        r[i] = ri;
        pp[i] = ri;
        pR[i] = (Real)ri;
        a2[0] += rhs * rhs;
        a2[1] += ri * ri;
        a2[2] += S[i] * ri;
    }
    if (p.tape_v) {
        double *tS = p.tape_v + (((size_t)s * p.N + (p.level - 1)) * 2 + 0) * p.ld;
        #pragma unroll 4
        for (int i = threadIdx.x; i < p.ld; i += blockDim.x) tS[i] = S[i];
    }
    block_sum(a2, sm);
    if (threadIdx.x == 0) {
        if (p.newton_level >= 0 && p.tr_newton)
            p.tr_newton[(size_t)s * p.N + p.newton_level] = st.newton_max;
        st.c = cp + st.yref;
        st.lambda = lambda;
        st.invW = invW;
        if (p.tape_s) {
            double *ts = p.tape_s + ((size_t)s * p.N + (p.level - 1)) * 4;
            ts[0] = lambda;
            ts[1] = invW;
        }
        st.rhs2 = a2[0];
        st.rr = a2[1];
        st.sp = a2[2];
        st.iters = 0;
        st.done = (a2[1] <= p.cg_tol2 * a2[0]) ? 1 : 0;
    }
}

// Four consecutive values at a 16-byte aligned address (two 16-byte accesses for doubles,
// one for floats).
__device__ __forceinline__ void ld4(double (&v)[4], const double *q)
{
    const double2 a = *reinterpret_cast<const double2 *>(q);
    const double2 b = *reinterpret_cast<const double2 *>(q + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st4(double *q, const double (&v)[4])
{
    *reinterpret_cast<double2 *>(q) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2 *>(q + 2) = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void st4(float *q, const float (&v)[4])
{
    *reinterpret_cast<float4 *>(q) = make_float4(v[0], v[1], v[2], v[3]);
}

// One pass of the CG iteration of Chronopoulos and Gear (1989), the form of conjugate
// gradients with a single reduction phase per iteration.  The product w = A r and the
// shares of delta = w . r come from k_reduce_partials; every block adds the shares in
// the same order and derives the pass's scalars (gamma = r . r):
//   t = 0: beta = 0, a = gamma / delta;
//   t > 0: beta = gamma / gamma_prev, a = gamma / (delta - beta gamma / a_prev),
// then
//   p = r + beta p,  s = w + beta s (= A p),  x += a p,  r -= a s,
// one warp per tile of kRedTile elements (four consecutive elements per lane), with the
// tile's shares of S . r and r . r for the next pass.  The last block of the query to
// finish (arrival counter) adds those shares, stores the new state and tests convergence;
// a query that is done stays done, so every block of a launch sees the same state.  Each
// FP64 warp instruction occupies the SM's FP64 pipe for many cycles on this part, so the
// scalar work is done once per query (in the reduction) rather than once per block.  In a
// CUDA graph (use_h = 1) the last query to finish sets the while-loop condition: 1 while
// some query has not converged and fewer than cg_max_iter passes ran (with one query,
// its last block does so without the second arrival).  Grid (nblk, Q).
template <typename Real>
__global__ void __launch_bounds__(32) k_cg_update(Params p, cudaGraphConditionalHandle h, int use_h)
{
    const int s = blockIdx.y, lane = threadIdx.x;
    SolveState &st = p.st[s];
    bool global_arrive = false;
    if (st.done) {
        global_arrive = blockIdx.x == 0;   // one block answers for a finished query
    } else {
        const WS<Real> ws(p);
        double *x = ws.v64(s, 0), *r = ws.v64(s, 1), *pp = ws.v64(s, 2), *S = ws.v64(s, 3),
               *w = ws.v64(s, 5), *sv = ws.v64(s, 7);
        Real *rR = ws.vR(s, 0);
        double *bp = p.bpart + (size_t)s * p.nblk * kBpart;
        const int t = st.iters;
        const double gam = st.rr;
        const int i0 = blockIdx.x * kRedTile + 4 * lane;
        const bool in = i0 < p.ld;   // ld is a multiple of 4
        // every value of the lane's four elements is loaded first, before the pass's scalars
        // are derived and before the first store (the vectors may alias as far as the
        // compiler can tell, so it would not move a later element's loads above a store)
        double rv[4], wv[4], pv[4], svv[4], xv[4], Sv[4];
        if (in) {
            ld4(rv, r + i0);
            ld4(wv, w + i0);
            ld4(xv, x + i0);
            ld4(Sv, S + i0);
            if (t > 0) {
                ld4(pv, pp + i0);
                ld4(svv, sv + i0);
            }
        }
        double dl = 0.0;   // delta = w . r: the shares in a fixed order, the same in every block
        for (int b = lane; b < p.nblk; b += 32) dl += __ldcg(bp + (size_t)b * kBpart);
#pragma unroll
        for (int o = 16; o; o >>= 1) dl += __shfl_xor_sync(0xffffffffu, dl, o);
        double beta = 0.0, den = dl;
        if (t > 0) {
            beta = gam / st.rr_prev;
            den = dl - beta * gam / st.cg_alpha;
        }
        const double a = gam / den;
        const int ok = (den > 0.0 && isfinite(a)) ? 1 : 0;
        double sr = 0.0, rr = 0.0;
        if (ok && in) {
            Real rn4[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const double pi = t > 0 ? rv[e] + beta * pv[e] : rv[e];
                const double si = t > 0 ? wv[e] + beta * svv[e] : wv[e];
                pv[e] = pi;
                svv[e] = si;
                xv[e] += a * pi;
                const double rn = rv[e] - a * si;
                rv[e] = rn;
                rn4[e] = (Real)rn;
                sr += Sv[e] * rn;
                rr += rn * rn;
            }
            st4(pp + i0, pv);
            st4(sv + i0, svv);
            st4(x + i0, xv);
            st4(r + i0, rv);
            st4(rR + i0, rn4);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            sr += __shfl_xor_sync(0xffffffffu, sr, o);
            rr += __shfl_xor_sync(0xffffffffu, rr, o);
        }
        int last = 0;
        if (lane == 0) {
            bp[(size_t)blockIdx.x * kBpart + 1] = sr;
            bp[(size_t)blockIdx.x * kBpart + 2] = rr;
            __threadfence();
            last = atomicAdd(&st.arrive_q, 1) == p.nblk - 1;
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        if (last) {
            __threadfence();
            double c0 = 0.0, c1 = 0.0;
            for (int b = lane; b < p.nblk; b += 32) {
                c0 += __ldcg(bp + (size_t)b * kBpart + 1);
                c1 += __ldcg(bp + (size_t)b * kBpart + 2);
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                c0 += __shfl_xor_sync(0xffffffffu, c0, o);
                c1 += __shfl_xor_sync(0xffffffffu, c1, o);
            }
            if (lane == 0) {
                st.arrive_q = 0;
                if (!ok) {  // breakdown: keep the current iterate
                    st.done = 1;
                    if (!(gam <= p.cg_tol2 * st.rhs2) && st.status == 0) st.status = FBSDE_ERR_CG;
                } else {
                    st.rr_prev = gam;
                    st.cg_alpha = a;
                    st.rr = c1;
                    st.sp = c0;
                    st.iters = t + 1;
                    st.cg_total += 1;
                    if (c1 <= p.cg_tol2 * st.rhs2) {
                        st.done = 1;
                    } else if (t + 1 >= p.cg_max_iter) {
                        st.done = 1;
                        st.cg_exhausted += 1;
                        if (st.status == 0) st.status = FBSDE_ERR_CG;
                    }
                }
                global_arrive = true;
            }
        }
    }
    if (use_h && global_arrive && lane == 0) {
        bool last_q = true;   // one query: its last block is the last arrival
        if (p.Q > 1) {
            __threadfence();
            last_q = atomicAdd(&p.st[0].arrive, 1) == p.Q - 1;
        }
        if (last_q) {
            if (p.Q > 1) __threadfence();
            p.st[0].arrive = 0;
            const int count = ++p.st[0].loop_iter;
            bool active = false;
            for (int q2 = 0; q2 < p.Q && !active; ++q2)
                active = *reinterpret_cast<volatile int *>(&p.st[q2].done) == 0;
            if (count >= p.cg_max_iter) active = false;
            cudaGraphSetConditional(h, active ? 1u : 0u);
        }
    }
}

// After the CG solve of level k: alpha = c - S . alpha_x (Eq. 3.20), Z_k = sigma alpha_x,
// trace outputs; at k = 0 the Newton step at x0 gives u(0,x0) (Algorithm 1).  The
// starting guess of the next level's solve is the linear extrapolation in k of the last
// two levels' alpha_x, g = 2 alpha_x^k - alpha_x^{k+1} (alpha_x^k alone at the top level):
// it starts the CG closer to the solution than alpha_x^k does (the solutions drift
// smoothly from level to level) and changes only the number of CG passes.
template <typename Real>
__global__ void __launch_bounds__(kFinThreads) k_cg_post(Params p)
{
    __shared__ double sm[32 * 4];
    const int s = blockIdx.x, k = p.level;
    const WS<Real> ws(p);
    SolveState &st = p.st[s];
    double *x = ws.v64(s, 0), *xp = ws.v64(s, 8);
    const double *S = ws.v64(s, 3);
    Real *xR = ws.vR(s, 1), *gR = ws.vR(s, 3);
    const bool extrap = k + 1 < p.N;   // alpha_x of level k+1 is in slot 8
    // S . alpha_x, sum alpha_x, |alpha_x|^2; forward SDE: alpha_x . x0, alpha_x . c_k
    double a[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const double *x0v = ws.v64(s, 6);
    const Real *ck = p.sde ? ws.anchor(s, k) : nullptr;
    #pragma unroll 4
    for (int i = threadIdx.x; i < p.ld; i += blockDim.x) {
        const double xi = x[i];
        const double g = extrap ? 2.0 * xi - xp[i] : xi;
        xp[i] = xi;
        x[i] = g;
        gR[i] = (Real)g;
        xR[i] = (Real)xi;
        a[0] += S[i] * xi;
        a[1] += xi;
        a[2] += xi * xi;
        if (ck) {
            a[3] += xi * x0v[i];
            a[4] += xi * (double)ck[i];
        }
        if (i < p.d) {
            if (p.tr_alpha_x) p.tr_alpha_x[((size_t)s * p.N + k) * p.d + i] = xi;
            if (k == 0 && p.grad) p.grad[(size_t)s * p.d + i] = xi;
        }
        if (p.tape_v) p.tape_v[(((size_t)s * p.N + k) * 2 + 1) * p.ld + i] = xi;
    }
    block_sum(a, sm);
    if (threadIdx.x == 0) {
        const double alpha = st.c - a[0];
        st.alpha = alpha;
        st.yref = alpha;
        st.sumz = p.sigma * a[1];
        st.zz = p.sigma * p.sigma * a[2];
        st.sum_ax = a[1];
        st.ax_x0 = a[3];
        st.newton_max = 0;
        // the traced intercept is the model's value at the anchor (D = 0): with a drift the
        // rows are centred at x0, so the intercept there moves by alpha_x . c_k
        if (p.tr_alpha) p.tr_alpha[(size_t)s * p.N + k] = alpha + a[4];
        if (p.tape_s) p.tape_s[((size_t)s * p.N + k) * 4 + 2] = alpha;
        if (p.tr_cg) p.tr_cg[(size_t)s * p.N + k] = st.iters;
        if (k == 0) {
            // every particle of level 0 sits at x0 (Delta_0 = 0): one Newton solve; with a
            // drift the prediction is taken at x0 + mu(x0) dt and sum_i z_i at sigma(x0)
            double E_hat = alpha, sumz = st.sumz;
            if (p.sde) {
                E_hat += p.dt * (p.mu0 * a[1] + p.mu1 * a[3]);
                sumz += p.sig1 * a[3];
            }
            const double feat = f_feature(p, 0.0, st.phi0, sumz, st.zz, st.psi0);
            int it;
            const double u = newton(p, E_hat, feat, it);
            if (it < 0 && st.status == 0) st.status = FBSDE_ERR_NEWTON;
            const int used = it < 0 ? p.newton_max_iter : it;
            st.newton_max_all = max(st.newton_max_all, used);
            if (p.tr_newton) p.tr_newton[(size_t)s * p.N] = used;
            if (!isfinite(u) && st.status == 0) st.status = FBSDE_ERR_NONFINITE;
            p.u0[s] = u;
        }
    }
}

// Before the CUDA-graph while loop around the CG passes: zero the pass counter and the
// arrival counter (kept in the first query's state) and set the loop condition to 1 only
// if some query still has to iterate, so a loop with nothing to do runs no pass.
template <typename Real> __global__ void k_cg_reset(Params p, cudaGraphConditionalHandle h)
{
    if (threadIdx.x != 0) return;
    p.st[0].loop_iter = 0;
    p.st[0].arrive = 0;
    bool active = false;
    for (int q = 0; q < p.Q && !active; ++q) active = p.st[q].done == 0;
    cudaGraphSetConditional(h, active ? 1u : 0u);
}

// Trace copy of the forward-sweep end state (X_N - x0 and Y_N) into FP64 arrays.
template <typename Real> __global__ void k_trace_forward(Params p)
{
    const WS<Real> ws(p);
    const int s = blockIdx.y;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < (size_t)p.M * p.d;
         idx += (size_t)gridDim.x * blockDim.x) {
        const long long j = idx / p.d;
        const int i = (int)(idx - (size_t)j * p.d);
        if (p.tr_x_N) p.tr_x_N[((size_t)s * p.M + j) * p.d + i] = (double)ws.row(s, j)[i];
        if (i == 0 && p.tr_y_N) p.tr_y_N[(size_t)s * p.M + j] = ws.Y(s)[j];
    }
}

template <typename Real>
__global__ void k_normals(uint64_t seed, uint32_t s, uint32_t k, uint32_t j0, int nj, int d, Real *out)
{
    constexpr int E = Chunk<Real>::E;
    const int nch = (d + E - 1) / E;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)nj * nch;
         idx += (long long)gridDim.x * blockDim.x) {
        const int jj = (int)(idx / nch), c = (int)(idx - (long long)jj * nch);
        const Chunk<Real> z = normal_chunk((Chunk<Real> *)nullptr, c, j0 + (uint32_t)jj, k, s, k0, k1, d);
#pragma unroll
        for (int e = 0; e < E; ++e)
            if (c * E + e < d) out[(size_t)jj * d + c * E + e] = z.v[e];
    }
}

}  // namespace dev
}  // namespace fbsde
