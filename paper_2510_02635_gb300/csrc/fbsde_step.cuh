// fbsde_step.cuh -- the fused per-level step of the FP32 path: one pass over the particle
// rows that draws the level's Brownian-bridge normals in registers, moves every row one
// level down (Eq. 2.7 walked backwards, reading R13), evaluates the local affine
// prediction, the driver f and the Newton iteration per particle (Eqs. 2.16-2.17), the
// Gaussian kernel weight of the next regression (Remark 2.3), and accumulates that
// regression's weighted d-vector moments (Eqs. 2.10-2.15) from the same rows.  8 bytes of
// HBM traffic per particle-dim: one read and one write of the row.  The terminal level
// (k = N) runs the same kernel without the read: the forward sweep's end point, g and the
// first regression's moments.  Included after fbsde_kernels.cuh.
//
// Block: kStepWarps consumer warps + one scalar warp (16 warps: 128 registers a thread).
// The CTA owns the contiguous rows [r0, r1) of one query, taken in stages of R rows
// (R in {1, 3, 5, 15, 30}, R * ld <= kStepElems floats where possible):
//   P1 (consumers)   team of T = 480 / R threads per row, VM chunks of 16 bytes each per
//                    thread: the chunks, loaded two ahead of their use through a register
//                    FIFO that runs on into the next stage, are stepped, written back to HBM and
//                    to a shared-memory slot; the four row sums (alpha_x . D, |D|^2,
//                    sum cos(x0 + D), g . D) go to shared memory per warp (or half-warp);
//   P2 (scalar warp) lane r handles row r of the stage: FP32 Newton, then FP64 Newton
//                    iterations that decide Y_k (the FP64 dependency chain is the latency
//                    that matters: 64 cycles per dependent FP64 operation on this part),
//                    the weight, the three moment coefficients; it runs while the
//                    consumers step the next stage;
//   P3 (consumers)   each thread owns fixed column chunks and adds the stage's rows,
//                    weighted by the three coefficients, into register accumulators.
// P3 of stage i-1 follows P1 of stage i, so P2 is off the consumers' critical path.
// Named barriers: A[b] "row sums of stage i ready" (consumers arrive, scalar warp
// waits), C[b] "coefficients of stage i ready" (scalar warp arrives, consumers wait),
// b = i mod 2.  Outputs: the updated rows, Y_k, the weights, per-CTA partial d-vectors
// (reduced by k_reduce_partials) and per-CTA scalar sums (spart).
#pragma once
#include "fbsde_kernels.cuh"

namespace fbsde {
namespace dev {

constexpr int kStepWarps = 15;   // + the scalar warp: 16 warps, four per SM sub-partition
constexpr int kStepConsumers = 32 * kStepWarps;
constexpr int kStepThreads = kStepConsumers + 32;
constexpr int kStepBarA = 1, kStepBarC = 3, kStepBarEnd = 5;

__device__ __forceinline__ void bar_arrive_named(int id, int nthreads)
{
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Philox words of one 16-byte chunk -> the four scaled normals scale * xi (Box-Muller
// pairs (0,1), (2,3)); bit-identical to normal_chunk for scale = 1.
__device__ __forceinline__ float4 normals_scaled(uint32_t c, uint32_t j, uint32_t k, uint32_t s,
                                                 uint32_t k0, uint32_t k1, float scale)
{
    const uint4 w = philox4x32_10(make_uint4(c, j, k, s), k0, k1);
    float4 z;
    box_muller_scaled(w.x, w.y, scale, z.x, z.y);
    box_muller_scaled(w.z, w.w, scale, z.z, z.w);
    return z;
}

__device__ __forceinline__ float dot4(float4 a, float4 b, float acc)
{
    acc = fmaf(a.x, b.x, acc);
    acc = fmaf(a.y, b.y, acc);
    acc = fmaf(a.z, b.z, acc);
    return fmaf(a.w, b.w, acc);
}

// Per-element term of the terminal feature sum in FP32 (g_term for Real = float).
__device__ __forceinline__ float g_term_f(int kind, float x, float th)
{
    switch (kind) {
    case FBSDE_AC_MANUFACTURED:
    case FBSDE_COS_LINEAR_TEST: return __cosf(x);
    case FBSDE_LOGISTIC_GRAD: return x;
    case FBSDE_HJB_LOGQUAD: return th * x * x;
    case FBSDE_AFFINE_TEST: return th * x;
    case FBSDE_AC_DOUBLEWELL: return x * x;
    default: return 0.0f;
    }
}

// f(y) and df/dy of the driver for a y-independent feature feat, in the arithmetic of T
// (the same table as f_scalar).
template <typename T>
__device__ __forceinline__ T f_of_y(int kind, T feat, T y, T c0, T c1, T lcoef, T &dfdy)
{
    switch (kind) {
    case FBSDE_AC_MANUFACTURED:
        dfdy = T(1) - T(3) * y * y;
        return y - y * y * y + feat;
    case FBSDE_LOGISTIC_GRAD:
        dfdy = feat;
        return (y - lcoef) * feat;
    case FBSDE_HJB_LOGQUAD:
        dfdy = T(0);
        return T(-0.5) * feat;
    case FBSDE_AFFINE_TEST:
        dfdy = c1;
        return c0 + c1 * y + feat;
    case FBSDE_COS_LINEAR_TEST:
        dfdy = c1;
        return c0 + c1 * y;
    case FBSDE_CUBIC_TEST:
    case FBSDE_AC_DOUBLEWELL:
        dfdy = T(1) - T(3) * y * y;
        return y - y * y * y;
    }
    dfdy = T(0);
    return T(0);
}

// Newton's iteration (2.17) on F(Y) = Y - E - dt f(Y) (2.16) with FP64 iterates: FP32
// Newton iterations first bring Y to within FP32 rounding of the root (cheap: an FP32
// operation has a short dependency latency), then FP64 iterations Y <- Y - F(Y) / F'
// with F evaluated in FP64 and F' taken at the FP32 iterate run until
// |dY| <= newton_tol max(1, |Y|), the stopping rule of the FP64 path.  The result is the
// FP64 root: F' only sets how fast each FP64 step contracts (its relative error is about
// 1e-7, so two FP64 steps from an FP32 root reach FP64 rounding).  feat_f / lc_f are the
// FP32 copies of the y-independent feature and of (2 + d) / (2d) (logistic driver),
// feat_d / lc_d the values the FP64 steps use.  iters = FP32 + FP64 iterations, or -1 if
// newton_max_iter ran out.
__device__ __forceinline__ double newton_fp32_fp64(const Params &p, double E, float feat_f,
                                                   double feat_d, float lc_f, double lc_d,
                                                   int &iters)
{
    const float c0 = (float)p.c0, c1 = (float)p.c1, dtf = (float)p.dt;
    const float Ef = (float)E;
    float yf = Ef;
    int n32 = 0;
    while (n32 < 8) {
        float dfdy;
        const float f = f_of_y<float>(p.kind, feat_f, yf, c0, c1, lc_f, dfdy);
        const float dy = __fdividef(yf - Ef - dtf * f, 1.0f - dtf * dfdy);
        yf -= dy;
        ++n32;
        if (!(fabsf(dy) > 2e-7f * fmaxf(1.0f, fabsf(yf)))) break;
    }
    float dfdy_f;
    (void)f_of_y<float>(p.kind, feat_f, yf, c0, c1, lc_f, dfdy_f);
    const double rdF = (double)__frcp_rn(1.0f - dtf * dfdy_f);
    double y = (double)yf;
    for (int m = 1; n32 + m <= p.newton_max_iter; ++m) {
        double dfdy;
        const double f = f_of_y<double>(p.kind, feat_d, y, p.c0, p.c1, lc_d, dfdy);
        const double dy = ((y - E) - p.dt * f) * rdF;
        y -= dy;
        if (fabs(dy) <= p.newton_tol * fmax(1.0, fabs(y))) {
            iters = n32 + m;
            return y;
        }
    }
    iters = -1;
    return y;
}

// Geometry of the fused step (host-computed, in Params): R rows per stage, T = 480 / R
// threads per row in P1 with VM chunks each (VM = ceil(nch / T), the template argument);
// P3 row groups of tpr threads (RG of them), vm3 <= VM chunks per thread; nslot
// shared-memory row slots.
template <int VM, bool COSF, bool TERM>
__global__ void __launch_bounds__(kStepThreads, 1) k_step(Params p)
{
    // chunks of the column pass held in registers; its sixth chunk (R = 1 with rows wider
    // than 9600 floats) accumulates in shared memory
    constexpr int VMR = VM < 5 ? VM : 5;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int g = blockIdx.x, s = blockIdx.y;
    const WS<float> ws(p);
    SolveState &st = p.st[s];
    constexpr bool terminal = TERM;
    const int ld = p.ld, nch = ld >> 2, d = p.d;
    const int R = p.st_R, T = p.st_T, nslot = p.st_nslot;
    float *vx = reinterpret_cast<float *>(smem_raw);   // alpha_x (terminal: unused)
    float *vg = vx + ld;                                // g (terminal: theta)
    float *vx0 = vg + ld;                               // x0
    float *slots = vx0 + ld;                            // [nslot][R][ld]
    const size_t slot_floats = (size_t)R * ld;
    float4 *wsum = reinterpret_cast<float4 *>(slots + p.st_region);   // [2][32]
    float4 *coef = wsum + 64;                                            // [2][32]
    float4 *tail = coef + 64;   // [3][nch - 5 kStepConsumers] column-pass chunks v = 5
    const bool has_tail = VM > 5 && p.st_vm3 > 5;   // only with R = 1 and nch > 2400
    const int ntail = has_tail ? nch - 5 * kStepConsumers : 0;
    for (int i = threadIdx.x; i < 3 * ntail; i += blockDim.x) tail[i] = make_float4(0.f, 0.f, 0.f, 0.f);

    const uint32_t sidx = p.solve0 + (uint32_t)s;
    for (int i = threadIdx.x; i < ld; i += blockDim.x) {
        vx[i] = terminal ? 0.0f : ws.vR(s, 1)[i];
        vg[i] = terminal ? ws.thetaR()[i] : ws.vR(s, 3)[i];
        vx0[i] = ws.vR(s, 2)[i];
    }
    __syncthreads();

    long long r0, r1;
    row_range(p.M, p.G, g, r0, r1);
    const int nst = (int)((r1 - r0 + R - 1) / R);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (warp == kStepWarps) {
        // ---------------- P2: the scalar warp ----------------
        const int PW = T >= 32 ? T >> 5 : 1;          // partial sums per row
        const double t_k = p.level * p.dt;
        const double rho_ref = p.sigma * p.sigma * p.d * t_k;
        const double wscale = -1.0 / (p.h2 * rho_ref);
        const float efac = COSF ? (float)(exp(t_k - p.T) / p.d) : 0.0f;
        const float acs = (float)(2.0 - 0.5 * p.sigma * p.sigma);
        const double lc_d = (2.0 + p.d) / (2.0 * p.d);
        const float lc_f = (float)lc_d;
        const double yref = terminal ? st.gx0 : st.alpha;
        const double feat_level = terminal ? 0.0 : f_feature(p, t_k, 0.0, st.sumz, st.zz);
        double accW = 0.0, accC = 0.0, accR = 0.0;
        int it_max = 0, failed = 0;
        for (int i = 0; i < nst; ++i) {
            const int b = i & 1;
            const long long base = r0 + (long long)i * R;
            const int nrows = (int)min((long long)R, r1 - base);
            bar_named(kStepBarA + b, kStepThreads);
            if (lane < nrows) {
                const long long j = base + lane;
                float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
                for (int w2 = 0; w2 < PW; ++w2) {
                    const float4 q = wsum[b * 32 + lane * PW + w2];
                    a0 += q.x;
                    a1 += q.y;
                    a2 += q.z;
                    a3 += q.w;
                }
                double Yj, rho;
                float gd = 0.0f;
                if (terminal) {
                    rho = (double)a0;
                    Yj = g_value(p, (double)a1);
                } else {
                    rho = (double)a1;
                    gd = a3;
                    float feat_f = (float)feat_level;
                    double feat_d = feat_level;
                    if (COSF) {   // the Allen-Cahn source at the particle, padding cos(0) removed
                        const float us = efac * (a2 - (float)(ld - d));
                        feat_f = us * us * us - acs * us;
                        feat_d = (double)feat_f;
                    }
                    int it;
                    Yj = newton_fp32_fp64(p, st.alpha + (double)a0, feat_f, feat_d, lc_f, lc_d, it);
                    if (it < 0) {
                        failed = 1;
                        it = p.newton_max_iter;
                    }
                    it_max = max(it_max, it);
                }
                const float wr = p.uniform ? 1.0f : expf((float)((rho - rho_ref) * wscale));
                const double dY = Yj - yref;
                coef[b * 32 + lane] = make_float4(wr, (float)((double)wr * dY), wr * gd, 0.0f);
                ws.Y(s)[j] = Yj;
                ws.w(s)[j] = wr;
                if (p.tape_w) {
                    p.tape_Y[((size_t)p.level * p.Q + s) * p.M + j] = Yj;
                    reinterpret_cast<float *>(p.tape_w)[((size_t)(p.level - 1) * p.Q + s) * p.M + j] = wr;
                }
                const double wd = (double)wr;
                accW += wd;
                accC = fma(wd, dY, accC);
                accR = fma(wd, rho, accR);
            }
            __syncwarp();
            bar_arrive_named(kStepBarC + b, kStepThreads);
        }
        // per-CTA scalar sums in lane order (fixed), Newton statistics
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            accW += __shfl_xor_sync(0xffffffffu, accW, o);
            accC += __shfl_xor_sync(0xffffffffu, accC, o);
            accR += __shfl_xor_sync(0xffffffffu, accR, o);
            it_max = max(it_max, __shfl_xor_sync(0xffffffffu, it_max, o));
        }
        const bool any_failed = __any_sync(0xffffffffu, failed);
        if (lane == 0) {
            double *o = ws.spart(s, g);
            o[0] = accW;
            o[1] = accC;
            o[2] = accR;
            if (!terminal) {
                if (it_max) {
                    atomicMax(&st.newton_max, it_max);
                    atomicMax(&st.newton_max_all, it_max);
                }
                if (any_failed) atomicCAS(&st.status, 0, (int)FBSDE_ERR_NEWTON);
            }
        }
        return;
    }

    // ---------------- consumers: P1 and P3 ----------------
    const int ct = threadIdx.x;                 // 0 .. kStepConsumers - 1
    const int team = ct / T, tl = ct - team * T;
    const int red_from = T >= 32 ? 16 : (T >> 1);
    const int pidx = T >= 32 ? warp : (ct >> 4);   // partial-sum slot of this (half-)warp
    const bool writer = T >= 32 ? lane == 0 : (lane & 15) == 0;
    const int tpr = p.st_tpr, RG = p.st_RG, vm3 = p.st_vm3;
    const int rg = ct / tpr, tc = ct - rg * tpr;
    const float wa = (float)p.wa, wb = (float)p.wb;
    const uint32_t kk = (uint32_t)p.level;
    float4 acc[3][VMR];
#pragma unroll
    for (int v = 0; v < VMR; ++v)
        acc[0][v] = acc[1][v] = acc[2][v] = make_float4(0.f, 0.f, 0.f, 0.f);
    // The rows this thread reads, Delta_{k+1}: chunk v of stage i sits at FIFO position
    // i VM + v; cur / nxt hold positions q and q + 1 while position q is stepped, and the
    // load of position q + 2 is issued then.  row_of(i) is the team's row of stage i, or
    // null past the CTA's rows.
    // row_of(i): the team's row of stage i, or null past the CTA's rows; the row of stage
    // i + a is a R ld floats further on.
    auto row_of = [&](int i) -> const float4 * {
        const long long j = r0 + (long long)i * R + team;
        return (!terminal && i < nst && j < r1) ? reinterpret_cast<const float4 *>(ws.row(s, j))
                                                : nullptr;
    };
    const int stage_chunks = R * (ld >> 2);
    float4 cur = make_float4(0.f, 0.f, 0.f, 0.f), nxt = cur;
    {
        const float4 *q0 = row_of(0), *q1 = row_of(VM > 1 ? 0 : 1);
        const int c0 = tl, c1 = tl + T * (VM > 1 ? 1 : 0);
        if (q0 && c0 < nch) cur = __ldcs(q0 + c0);
        if (q1 && c1 < nch) nxt = __ldcs(q1 + c1);
    }

    auto p3 = [&](int i) {
        const int b = i & 1;
        const long long base = r0 + (long long)i * R;
        const int nrows = (int)min((long long)R, r1 - base);
        bar_named(kStepBarC + b, kStepThreads);
        if (rg < RG) {
            const float *sl = slots + (size_t)(i % nslot) * slot_floats;
            for (int r = rg; r < nrows; r += RG) {
                const float4 cf = coef[b * 32 + r];
                const float4 *row = reinterpret_cast<const float4 *>(sl + (size_t)r * ld);
                if (VM > 5 && has_tail) {
                    const int c = tc + tpr * 5;
                    if (c < nch) {
                        const float4 x = row[c];
                        float4 *t0 = tail + (c - 5 * kStepConsumers);
                        float4 a0 = t0[0], a1 = t0[ntail], a2 = t0[2 * ntail];
                        a0.x = fmaf(cf.x, x.x, a0.x);
                        a0.y = fmaf(cf.x, x.y, a0.y);
                        a0.z = fmaf(cf.x, x.z, a0.z);
                        a0.w = fmaf(cf.x, x.w, a0.w);
                        a1.x = fmaf(cf.y, x.x, a1.x);
                        a1.y = fmaf(cf.y, x.y, a1.y);
                        a1.z = fmaf(cf.y, x.z, a1.z);
                        a1.w = fmaf(cf.y, x.w, a1.w);
                        a2.x = fmaf(cf.z, x.x, a2.x);
                        a2.y = fmaf(cf.z, x.y, a2.y);
                        a2.z = fmaf(cf.z, x.z, a2.z);
                        a2.w = fmaf(cf.z, x.w, a2.w);
                        t0[0] = a0;
                        t0[ntail] = a1;
                        t0[2 * ntail] = a2;
                    }
                }
#pragma unroll
                for (int v = 0; v < VMR; ++v) {
                    const int c = tc + tpr * v;
                    if (v < vm3 && c < nch) {
                        const float4 x = row[c];
                        acc[0][v].x = fmaf(cf.x, x.x, acc[0][v].x);
                        acc[0][v].y = fmaf(cf.x, x.y, acc[0][v].y);
                        acc[0][v].z = fmaf(cf.x, x.z, acc[0][v].z);
                        acc[0][v].w = fmaf(cf.x, x.w, acc[0][v].w);
                        acc[1][v].x = fmaf(cf.y, x.x, acc[1][v].x);
                        acc[1][v].y = fmaf(cf.y, x.y, acc[1][v].y);
                        acc[1][v].z = fmaf(cf.y, x.z, acc[1][v].z);
                        acc[1][v].w = fmaf(cf.y, x.w, acc[1][v].w);
                        acc[2][v].x = fmaf(cf.z, x.x, acc[2][v].x);
                        acc[2][v].y = fmaf(cf.z, x.y, acc[2][v].y);
                        acc[2][v].z = fmaf(cf.z, x.z, acc[2][v].z);
                        acc[2][v].w = fmaf(cf.z, x.w, acc[2][v].w);
                    }
                }
            }
        }
    };

    for (int i = 0; i < nst; ++i) {
        const int b = i & 1;
        const long long base = r0 + (long long)i * R;
        const int nrows = (int)min((long long)R, r1 - base);
        const long long j = base + team;
        float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
        float4 *dst = reinterpret_cast<float4 *>(ws.row(s, team < nrows ? j : base));
        float4 *sl = reinterpret_cast<float4 *>(slots + (size_t)(i % nslot) * slot_floats +
                                                (size_t)team * ld);
        if (terminal) {
            if (team < nrows) {
                const int kind = p.kind;
#pragma unroll
                for (int v = 0; v < VM; ++v) {
                    const int c = tl + T * v;
                    if (c < nch) {
                        float4 z = normals_scaled((uint32_t)c, (uint32_t)j, kk, sidx, p.key0,
                                                  p.key1, wb);
                        const float4 x0c = reinterpret_cast<const float4 *>(vx0)[c];
                        const float4 thc = reinterpret_cast<const float4 *>(vg)[c];
                        const int i0 = 4 * c;
                        if (i0 + 1 >= d) z.y = 0.0f;
                        if (i0 + 2 >= d) z.z = 0.0f;
                        if (i0 + 3 >= d) z.w = 0.0f;
                        s0 = dot4(z, z, s0);
                        s1 += g_term_f(kind, x0c.x + z.x, thc.x);
                        if (i0 + 1 < d) s1 += g_term_f(kind, x0c.y + z.y, thc.y);
                        if (i0 + 2 < d) s1 += g_term_f(kind, x0c.z + z.z, thc.z);
                        if (i0 + 3 < d) s1 += g_term_f(kind, x0c.w + z.w, thc.w);
                        sl[c] = z;
                        __stcs(dst + c, z);
                    }
                }
            }
        } else {
            const float4 *ahead0 = row_of(i);
            const bool has1 = i + 1 < nst && j + R < r1, has2 = i + 2 < nst && j + 2 * R < r1;
#pragma unroll
            for (int v = 0; v < VM; ++v) {
                const int c = tl + T * v;
                const float4 dold = cur;
                cur = nxt;
                {   // load FIFO position i VM + v + 2
                    const int vq = (v + 2) % VM, iq = (v + 2) / VM;
                    const bool has = iq == 0 ? (ahead0 != nullptr) : (iq == 1 ? has1 : has2);
                    const int cq = tl + T * vq;
                    if (has && cq < nch) nxt = __ldcs(ahead0 + (size_t)iq * stage_chunks + cq);
                }
                if (team < nrows && c < nch) {
                    float4 z = normals_scaled((uint32_t)c, (uint32_t)j, kk, sidx, p.key0,
                                              p.key1, wb);
                    if (4 * c + 4 > d) {   // the row's last chunk: padding stays zero
                        const int i0 = 4 * c;
                        if (i0 + 1 >= d) z.y = 0.0f;
                        if (i0 + 2 >= d) z.z = 0.0f;
                        if (i0 + 3 >= d) z.w = 0.0f;
                    }
                    float4 dn;
                    dn.x = fmaf(wa, dold.x, z.x);
                    dn.y = fmaf(wa, dold.y, z.y);
                    dn.z = fmaf(wa, dold.z, z.z);
                    dn.w = fmaf(wa, dold.w, z.w);
                    const float4 ax = reinterpret_cast<const float4 *>(vx)[c];
                    const float4 gg = reinterpret_cast<const float4 *>(vg)[c];
                    s0 = dot4(ax, dn, s0);
                    s1 = dot4(dn, dn, s1);
                    s3 = dot4(gg, dn, s3);
                    if (COSF) {
                        const float4 xc = reinterpret_cast<const float4 *>(vx0)[c];
                        s2 += (__cosf(xc.x + dn.x) + __cosf(xc.y + dn.y)) +
                              (__cosf(xc.z + dn.z) + __cosf(xc.w + dn.w));
                    }
                    sl[c] = dn;
                    __stcs(dst + c, dn);
                }
            }
        }
        for (int o = red_from; o; o >>= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
            s3 += __shfl_xor_sync(0xffffffffu, s3, o);
        }
        if (writer) wsum[b * 32 + pidx] = make_float4(s0, s1, s2, s3);
        __syncwarp();
        bar_arrive_named(kStepBarA + b, kStepThreads);
        if (i >= 1) p3(i - 1);
    }
    if (nst >= 1) p3(nst - 1);

    // per-CTA partial d-vectors: row groups summed in group order (threads past the RG
    // row groups of tpr threads own no chunk)
    if (RG == 1) {
        if (rg >= RG) return;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float4 *dst = reinterpret_cast<float4 *>(ws.part(s, g, a));
#pragma unroll
            for (int v = 0; v < VMR; ++v) {
                const int c = tc + tpr * v;
                if (v < vm3 && c < nch) dst[c] = acc[a][v];
            }
            if (VM > 5 && has_tail) {
                const int c = tc + tpr * 5;
                if (c < nch) dst[c] = tail[a * ntail + (c - 5 * kStepConsumers)];
            }
        }
        return;
    }
    bar_named(kStepBarEnd, kStepConsumers);   // every consumer is past its last slot read
    float4 *red = reinterpret_cast<float4 *>(slots);  // [RG][3][nch]
    if (rg < RG) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (tc < nch) red[((size_t)rg * 3 + a) * nch + tc] = acc[a][0];
    }
    bar_named(kStepBarEnd, kStepConsumers);
    for (int idx = ct; idx < 3 * nch; idx += kStepConsumers) {
        const int a = idx / nch, c = idx - a * nch;
        float4 sum = red[(size_t)a * nch + c];
        for (int r = 1; r < RG; ++r) {
            const float4 o = red[((size_t)r * 3 + a) * nch + c];
            sum.x += o.x;
            sum.y += o.y;
            sum.z += o.z;
            sum.w += o.w;
        }
        reinterpret_cast<float4 *>(ws.part(s, g, a))[c] = sum;
    }
}

}  // namespace dev
}  // namespace fbsde
