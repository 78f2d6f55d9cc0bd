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
// Block: kStepWarps consumer warps + one service warp (16 warps: 128 registers a thread).
// The CTA owns the contiguous rows [r0, r1) of one query, taken in stages of R rows
// (R in {1, 3, 5, 15, 30}, R * ld <= kStepElems floats where possible):
//   load (service warp, one lane)  the rows Delta_{k+1} of stage i + 2 are copied into a
//                    two-slot shared-memory ring by one bulk copy (cp.async.bulk, completion
//                    on the slot's mbarrier) as soon as the consumers are done with stage i;
//   P1 (consumers)   team of T = 480 / R threads per row, VM chunks of 16 bytes each per
//                    thread: the chunks are read from the ring, stepped and written back to
//                    HBM; the four row sums (alpha_x . D, |D|^2, sum cos(x0 + D), g . D) go
//                    to shared memory per warp (or half-warp);
//   P2 (service warp) lane r handles row r of the stage: FP32 Newton, then FP64 Newton
//                    iterations that decide Y_k (the FP64 dependency chain is the latency
//                    that matters: 64 cycles per dependent FP64 operation on this part),
//                    the weight, the three moment coefficients; it runs while the
//                    consumers step the next stage;
//   P3 (consumers)   each thread owns fixed column chunks and adds the stage's updated rows,
//                    read back from L2 (they were written one stage earlier), weighted by
//                    the three coefficients, into register accumulators.
// P3 of stage i-1 follows P1 of stage i, so P2 is off the consumers' critical path.
// Hand-offs by mbarriers (b = i mod 2): sums[b] "stage i stepped: row sums written, ring
// slot free" (every consumer arrives, the service warp waits), coefb[b] "coefficients of
// stage i ready" (the service warp arrives, each consumer waits on its own), so the
// consumer warps never wait for one another and a fast warp may run a stage ahead.  Outputs: the updated rows, Y_k, the weights,
// per-CTA partial d-vectors (reduced by k_reduce_partials) and per-CTA scalar sums (spart).
#pragma once
#include "fbsde_matvec.cuh"   // mbarrier and bulk-copy helpers

namespace fbsde {
namespace dev {

constexpr int kStepWarps = 15;   // + the scalar warp: 16 warps, four per SM sub-partition
constexpr int kStepConsumers = 32 * kStepWarps;
constexpr int kStepThreads = kStepConsumers + 32;
constexpr int kStepBarEnd = 5;   // named barrier of the consumers' final reduction

// Philox words of one 16-byte chunk -> the four scaled normals scale * xi (Box-Muller
// pairs (0,1), (2,3)); bit-identical to normal_chunk for scale = 1.
__device__ __forceinline__ float4 normals_scaled(const Params &p, uint32_t c, uint32_t j,
                                                 uint32_t k, uint32_t s, float scale)
{
    const uint4 w = philox4x32_10_rk(make_uint4(c, j, k, s), p.rk0, p.rk1);
    float4 z;
    box_muller_scaled(w.x, w.y, scale, z.x, z.y);
    box_muller_scaled(w.z, w.w, scale, z.z, z.w);
    return z;
}

// Sum of the four row sums over a warp, scattered: afterwards lanes 8q .. 8q + 7 hold the
// warp's total of value q (q = 0..3).  Six shuffles instead of twenty: the first two
// exchanges halve the values each lane carries, the last three sum the one left.
__device__ __forceinline__ float warp_sum4_scatter(float s0, float s1, float s2, float s3, int lane)
{
    const bool hi16 = lane & 16, hi8 = lane & 8;
    float k0 = hi16 ? s2 : s0, k1 = hi16 ? s3 : s1;
    const float o0 = hi16 ? s0 : s2, o1 = hi16 ? s1 : s3;
    k0 += __shfl_xor_sync(0xffffffffu, o0, 16);
    k1 += __shfl_xor_sync(0xffffffffu, o1, 16);
    float k = hi8 ? k1 : k0;
    const float o = hi8 ? k0 : k1;
    k += __shfl_xor_sync(0xffffffffu, o, 8);
    k += __shfl_xor_sync(0xffffffffu, k, 4);
    k += __shfl_xor_sync(0xffffffffu, k, 2);
    k += __shfl_xor_sync(0xffffffffu, k, 1);
    return k;
}

// a * b + c on both halves of a pair at once: the packed FP32 fused multiply-add of this
// architecture (one instruction for two FMAs)
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }
// acc + a . b over the four components, as two pairs
__device__ __forceinline__ float2 dot4x2(float4 a, float4 b, float2 acc)
{
    return fma2(hi2(a), hi2(b), fma2(lo2(a), lo2(b), acc));
}

__device__ __forceinline__ float dot4(float4 a, float4 b, float acc)
{
    acc = fmaf(a.x, b.x, acc);
    acc = fmaf(a.y, b.y, acc);
    acc = fmaf(a.z, b.z, acc);
    return fmaf(a.w, b.w, acc);
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
// P3 row groups of tpr threads (RG of them), vm3 <= VM chunks per thread.  ONE: the
// one-row stage (R = 1, T = tpr = 480, rows wider than
// 3413 floats) with its strides known at compile time; its chunks v < VM - 1 always lie
// inside the row.
template <int VM, bool COSF, bool TERM, bool ONE>
__global__ void __launch_bounds__(kStepThreads, 1) k_step(Params p)
{
    // chunks of the column pass held in registers; its sixth chunk (R = 1 with rows wider
    // than 9600 floats) accumulates in shared memory
    constexpr int VMR = VM < 5 ? VM : 5;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int g = blockIdx.x, s = blockIdx.y;
    const WS<float> ws(p);
    SolveState &st = p.st[s];
    constexpr bool terminal = TERM;
    const int ld = p.ld, nch = ld >> 2, d = p.d;
    const int R = ONE ? 1 : p.st_R, T = ONE ? kStepConsumers : p.st_T;
    float *vx = reinterpret_cast<float *>(smem_raw);   // alpha_x (terminal: unused)
    float *vg = vx + ld;                                // g (terminal: theta)
    float *vx0 = vg + ld;                               // x0
    float *ring = vx0 + ld;                             // [2][R][ld] rows Delta_{k+1}
    const size_t slot_floats = (size_t)R * ld;
    float4 *wsum = reinterpret_cast<float4 *>(ring + p.st_region);    // [2][32]
    float4 *coef = wsum + 64;                                            // [2][32]
    // mbarriers: full[2] ring slot loaded (bulk-copy bytes), sums[2] row sums of a stage
    // written by every consumer thread, coefb[2] coefficients of a stage written by the
    // service warp; slot / buffer b = stage mod 2
    uint64_t *full = reinterpret_cast<uint64_t *>(coef + 64);
    uint64_t *sums = full + 2, *coefb = full + 4;
    float4 *tail = reinterpret_cast<float4 *>(full + 6);  // [3][nch - 5 kStepConsumers]
    const bool has_tail = VM > 5 && p.st_vm3 > 5;   // only with R = 1 and nch > 2400
    const int ntail = has_tail ? nch - 5 * kStepConsumers : 0;
    for (int i = threadIdx.x; i < 3 * ntail; i += blockDim.x) tail[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (threadIdx.x == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&sums[b], kStepConsumers);
            mbar_init(&coefb[b], 32);
        }
        fence_mbar_init();
    }

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

    bool timed_out = false;
    const uint32_t row_bytes = (uint32_t)ld * sizeof(float);
    // bulk copy of the rows of stage i into ring slot i mod 2 (one lane of the service warp)
    auto load_stage = [&](int i) {
        const long long base = r0 + (long long)i * R;
        const uint32_t rows = (uint32_t)min((long long)R, r1 - base);
        uint64_t *bar = &full[i & 1];
        mbar_arrive_expect_tx(bar, rows * row_bytes);
        bulk_g2s(ring + (size_t)(i & 1) * slot_floats, ws.row(s, base), rows * row_bytes, bar);
    };

    if (warp == kStepWarps) {
        // ---------------- the service warp: ring loads and P2 ----------------
        if (!terminal && lane == 0) {
            if (nst > 0) load_stage(0);
            if (nst > 1) load_stage(1);
        }
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
        const bool cos_g = p.kind == FBSDE_AC_MANUFACTURED || p.kind == FBSDE_COS_LINEAR_TEST;
        double accW = 0.0, accC = 0.0, accR = 0.0;
        int it_max = 0, failed = 0;
        for (int i = 0; i < nst; ++i) {
            const int b = i & 1;
            const long long base = r0 + (long long)i * R;
            const int nrows = (int)min((long long)R, r1 - base);
            mbar_wait_or_flag(&sums[b], (uint32_t)((i >> 1) & 1), timed_out);
            // the consumers are done with slot i mod 2: refill it with stage i + 2
            if (!terminal && lane == 0 && i + 2 < nst) load_stage(i + 2);
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
                    Yj = g_value(p, (double)a1 - (cos_g ? (double)(ld - d) : 0.0));
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
            mbar_arrive(&coefb[b]);
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
        if (!terminal && lane == 0) {   // every copy issued has landed before the CTA exits
            for (int i = max(0, nst - 2); i < nst; ++i)
                mbar_wait_or_flag(&full[i & 1], (uint32_t)((i >> 1) & 1), timed_out);
        }
        if (timed_out) atomicCAS(&st.status, 0, (int)FBSDE_ERR_TIMEOUT);
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
    const int team = ONE ? 0 : ct / T, tl0 = ONE ? ct : ct - team * T;
    const int tpr = ONE ? kStepConsumers : p.st_tpr, RG = ONE ? 1 : p.st_RG;
    const int vm3 = ONE ? VM : p.st_vm3;
    const int rg = ONE ? 0 : ct / tpr, tc = ONE ? ct : ct - rg * tpr;
    const float wa = (float)p.wa, wb = (float)p.wb;
    const uint32_t kk = (uint32_t)p.level;
    // chunk v = tl + T v of a row exists (ONE: every v < VM - 1 does)
    auto in_row = [&](int v, int c) { return (ONE && v < VM - 1) || c < nch; };
    float4 acc[3][VMR];
#pragma unroll
    for (int v = 0; v < VMR; ++v)
        acc[0][v] = acc[1][v] = acc[2][v] = make_float4(0.f, 0.f, 0.f, 0.f);
    // fma of one chunk of a row into the three accumulators of chunk v
    auto acc3 = [&](float4 (&a)[3], const float4 cf, const float4 x) {
        const float2 xl = lo2(x), xh = hi2(x);
        const float2 c0 = make_float2(cf.x, cf.x), c1 = make_float2(cf.y, cf.y),
                     c2 = make_float2(cf.z, cf.z);
        float2 l = fma2(c0, xl, lo2(a[0])), h = fma2(c0, xh, hi2(a[0]));
        a[0] = make_float4(l.x, l.y, h.x, h.y);
        l = fma2(c1, xl, lo2(a[1]));
        h = fma2(c1, xh, hi2(a[1]));
        a[1] = make_float4(l.x, l.y, h.x, h.y);
        l = fma2(c2, xl, lo2(a[2]));
        h = fma2(c2, xh, hi2(a[2]));
        a[2] = make_float4(l.x, l.y, h.x, h.y);
    };
    auto p3 = [&](int i) {
        const int b = i & 1;
        const long long base = r0 + (long long)i * R;
        const int nrows = ONE ? 1 : (int)min((long long)R, r1 - base);
        if (ONE) {
            // the row stepped in P1 of stage i, read back through L2.  With one row per
            // stage the row pass and the column pass own the same chunks, so these are this
            // thread's own stores and the loads can be issued before the wait for the
            // stage's coefficients.
            const float4 *row = reinterpret_cast<const float4 *>(ws.row(s, base));
            float4 x[VM];
#pragma unroll
            for (int v = 0; v < VM; ++v) {
                const int c = tc + tpr * v;
                if (in_row(v, c)) x[v] = __ldcg(row + c);
            }
            mbar_wait_or_flag(&coefb[b], (uint32_t)((i >> 1) & 1), timed_out);
            const float4 cf = coef[b * 32];
#pragma unroll
            for (int v = 0; v < VMR; ++v) {
                float4 a[3] = {acc[0][v], acc[1][v], acc[2][v]};
                if (in_row(v, tc + tpr * v)) acc3(a, cf, x[v]);
                acc[0][v] = a[0];
                acc[1][v] = a[1];
                acc[2][v] = a[2];
            }
            if (VM > 5 && has_tail) {
                const int c = tc + tpr * 5;
                if (c < nch) {
                    float4 *t0 = tail + (c - 5 * kStepConsumers);
                    float4 a[3] = {t0[0], t0[ntail], t0[2 * ntail]};
                    acc3(a, cf, x[VM - 1]);
                    t0[0] = a[0];
                    t0[ntail] = a[1];
                    t0[2 * ntail] = a[2];
                }
            }
            return;
        }
        mbar_wait_or_flag(&coefb[b], (uint32_t)((i >> 1) & 1), timed_out);
        if (rg < RG) {
            for (int r = rg; r < nrows; r += RG) {
                const float4 cf = coef[b * 32 + r];
                // the row stepped in P1 of stage i, read back through L2
                const float4 *row = reinterpret_cast<const float4 *>(ws.row(s, base + r));
#pragma unroll
                for (int v = 0; v < VMR; ++v) {
                    const int c = tc + tpr * v;
                    if (v < vm3 && c < nch) {
                        float4 a[3] = {acc[0][v], acc[1][v], acc[2][v]};
                        acc3(a, cf, __ldcg(row + c));
                        acc[0][v] = a[0];
                        acc[1][v] = a[1];
                        acc[2][v] = a[2];
                    }
                }
            }
        }
    };

    for (int i = 0; i < nst; ++i) {
        const int b = i & 1;
        const long long base = r0 + (long long)i * R;
        const int nrows = ONE ? 1 : (int)min((long long)R, r1 - base);
        const bool active = ONE || team < nrows;
        const int tl = tl0;
        const long long j = base + team;
        float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
        float2 q0 = make_float2(0.f, 0.f), q1 = q0, q3 = q0;   // pair sums of the level step
        float4 *dst = reinterpret_cast<float4 *>(ws.row(s, active ? j : base));
        if (terminal) {
            if (active) {
                const int kind = p.kind;
#pragma unroll
                for (int v = 0; v < VM; ++v) {
                    const int c = tl + T * v;
                    if (in_row(v, c)) {
                        float4 z = normals_scaled(p, (uint32_t)c, (uint32_t)j, kk, sidx, wb);
                        if ((!ONE || v == VM - 1) && 4 * c + 4 > d) {   // padding stays 0
                            const int i0 = 4 * c;
                            if (i0 + 1 >= d) z.y = 0.0f;
                            if (i0 + 2 >= d) z.z = 0.0f;
                            if (i0 + 3 >= d) z.w = 0.0f;
                        }
                        s0 = dot4(z, z, s0);
                        // terminal feature of g at x0 + Delta_N (padding: x0 = theta = 0, so
                        // only the cosine kinds see it, as cos 0 = 1, removed in P2)
                        const float4 xc = reinterpret_cast<const float4 *>(vx0)[c];
                        const float4 x = make_float4(xc.x + z.x, xc.y + z.y, xc.z + z.z, xc.w + z.w);
                        if (kind == FBSDE_AC_MANUFACTURED || kind == FBSDE_COS_LINEAR_TEST) {
                            s1 += (cos_ftz(x.x) + cos_ftz(x.y)) + (cos_ftz(x.z) + cos_ftz(x.w));
                        } else if (kind == FBSDE_LOGISTIC_GRAD) {
                            s1 += (x.x + x.y) + (x.z + x.w);
                        } else if (kind == FBSDE_AC_DOUBLEWELL) {
                            s1 = dot4(x, x, s1);
                        } else if (kind == FBSDE_HJB_LOGQUAD || kind == FBSDE_AFFINE_TEST) {
                            const float4 th = reinterpret_cast<const float4 *>(vg)[c];
                            const float4 tx = make_float4(th.x * x.x, th.y * x.y, th.z * x.z,
                                                          th.w * x.w);
                            s1 = kind == FBSDE_HJB_LOGQUAD ? dot4(tx, x, s1)
                                                           : s1 + ((tx.x + tx.y) + (tx.z + tx.w));
                        }
                        dst[c] = z;
                    }
                }
            }
        } else {
            mbar_wait_or_flag(&full[b], (uint32_t)((i >> 1) & 1), timed_out);
            const float4 *sl = reinterpret_cast<const float4 *>(ring + (size_t)b * slot_floats +
                                                                (size_t)team * ld);
            if (active) {
#pragma unroll
                for (int v = 0; v < VM; ++v) {
                    const int c = tl + T * v;
                    if (in_row(v, c)) {
                        const float4 dold = sl[c];
                        float4 z = normals_scaled(p, (uint32_t)c, (uint32_t)j, kk, sidx, wb);
                        if ((!ONE || v == VM - 1) && 4 * c + 4 > d) {   // padding stays 0
                            const int i0 = 4 * c;
                            if (i0 + 1 >= d) z.y = 0.0f;
                            if (i0 + 2 >= d) z.z = 0.0f;
                            if (i0 + 3 >= d) z.w = 0.0f;
                        }
                        const float2 wa2 = make_float2(wa, wa);
                        const float2 dl = fma2(wa2, lo2(dold), lo2(z)),
                                     dh = fma2(wa2, hi2(dold), hi2(z));
                        const float4 dn = make_float4(dl.x, dl.y, dh.x, dh.y);
                        const float4 ax = reinterpret_cast<const float4 *>(vx)[c];
                        const float4 gg = reinterpret_cast<const float4 *>(vg)[c];
                        q0 = dot4x2(ax, dn, q0);
                        q1 = dot4x2(dn, dn, q1);
                        q3 = dot4x2(gg, dn, q3);
                        if (COSF) {
                            const float4 xc = reinterpret_cast<const float4 *>(vx0)[c];
                            const float2 xa = __fadd2_rn(lo2(xc), dl), xb = __fadd2_rn(hi2(xc), dh);
                            s2 += (cos_ftz(xa.x) + cos_ftz(xa.y)) + (cos_ftz(xb.x) + cos_ftz(xb.y));
                        }
                        dst[c] = dn;
                    }
                }
            }
            s0 += q0.x + q0.y;
            s1 += q1.x + q1.y;
            s3 += q3.x + q3.y;
        }
        if (T >= 32) {   // one partial per warp; lane 8q writes component q
            const float k4 = warp_sum4_scatter(s0, s1, s2, s3, lane);
            if ((lane & 7) == 0) reinterpret_cast<float *>(wsum + b * 32 + warp)[lane >> 3] = k4;
        } else {         // half-warp teams: one partial per half-warp
#pragma unroll
            for (int o = 8; o; o >>= 1) {
                s0 += __shfl_xor_sync(0xffffffffu, s0, o);
                s1 += __shfl_xor_sync(0xffffffffu, s1, o);
                s2 += __shfl_xor_sync(0xffffffffu, s2, o);
                s3 += __shfl_xor_sync(0xffffffffu, s3, o);
            }
            if ((lane & 15) == 0) wsum[b * 32 + (ct >> 4)] = make_float4(s0, s1, s2, s3);
        }
        mbar_arrive(&sums[b]);
        if (i >= 1) p3(i - 1);
    }
    if (nst >= 1) p3(nst - 1);
    if (timed_out) atomicCAS(&st.status, 0, (int)FBSDE_ERR_TIMEOUT);

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
                if (v < vm3 && in_row(v, c)) dst[c] = acc[a][v];
            }
            if (VM > 5 && has_tail) {
                const int c = tc + tpr * 5;
                if (c < nch) dst[c] = tail[a * ntail + (c - 5 * kStepConsumers)];
            }
        }
        return;
    }
    bar_named(kStepBarEnd, kStepConsumers);   // every consumer is past its last ring read
    float4 *red = reinterpret_cast<float4 *>(ring);   // [RG][3][nch]
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
