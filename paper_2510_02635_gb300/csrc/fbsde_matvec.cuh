// fbsde_matvec.cuh -- the matrix-free product of the regression operator (the dominant
// kernel of a solve), fed by bulk copies (TMA) through an mbarrier-synchronised
// shared-memory ring.  Included after fbsde_kernels.cuh.
#pragma once
#include "fbsde_kernels.cuh"

namespace fbsde {
namespace dev {

// ---------------------------------------------------------------------------
// mbarrier + bulk-copy (TMA) helpers.  Every wait is bounded: after kWaitNs of
// %globaltimer without completion it returns false and the caller records
// FBSDE_ERR_TIMEOUT instead of spinning forever.
// ---------------------------------------------------------------------------
constexpr unsigned long long kWaitNs = 5ull * 1000 * 1000 * 1000;

__device__ __forceinline__ uint32_t smem_u32(const void *ptr)
{
    return (uint32_t)__cvta_generic_to_shared(ptr);
}
__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n"
        "  .reg .pred q;\n"
        "  mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n"
        "  selp.u32 %0, 1, 0, q;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits for the completion of the barrier phase with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          unsigned long long limit_ns = kWaitNs)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer_ns() - t0 > limit_ns) return false;
    }
}
// Bounded wait whose failure is sticky: after the first timeout of this thread, later
// waits only poll once, so a broken pipeline costs one kWaitNs per thread, not one per
// stage.
__device__ __forceinline__ void mbar_wait_or_flag(uint64_t *bar, uint32_t parity, bool &timed_out,
                                                  unsigned long long limit_ns = kWaitNs)
{
    if (timed_out) {
        (void)mbar_try_wait(bar, parity);
        return;
    }
    if (!mbar_wait(bar, parity, limit_ns)) timed_out = true;
}

// Bulk copy global -> shared memory; completion is signalled on bar as transaction bytes.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// ---------------------------------------------------------------------------
// Matrix-free product of the regression (Sec. 2.4, Steps 1 and 2) on the centred
// operator: partial_g = sum_{j in CTA g} w_j (D_j . v) D_j with v = vR(s, 0).
// Warp 0 is the producer: one lane streams the CTA's rows, mv_rows consecutive rows
// (one contiguous block) per stage, into a ring of mv_stages shared-memory stages
// with cp.async.bulk, completion counted on the stage's "full" mbarrier.  The other
// warps form nteams consumer teams of team_warps warps; a team owns one row at a time:
// dot product from shared memory, team sum (warp butterfly + one named barrier),
// then the weighted row sum into register accumulators.  Each consumer warp arrives
// on the stage's "empty" mbarrier when done, which lets the producer refill it.
// ---------------------------------------------------------------------------
template <typename Real, int VPT, bool WIDE>
__global__ void __launch_bounds__(WIDE ? 544 : (VPT >= 8 ? 352 : 288), 1) k_matvec(Params p)
{
    constexpr int E = Chunk<Real>::E;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int g = blockIdx.x, s = blockIdx.y;
    if (p.st[s].done) return;
    const WS<Real> ws(p);
    const int nch = p.ld / E;
    const int S = p.mv_stages, R = p.mv_rows;
    const int tw = p.team_warps;
    const int nteams = (blockDim.x / 32 - 1) / tw;
    const size_t row_elems = (size_t)p.ld;
    const uint32_t row_bytes = (uint32_t)(row_elems * sizeof(Real));
    Real *ring = reinterpret_cast<Real *>(smem_raw);                     // [S][R][ld]
    uint64_t *full = reinterpret_cast<uint64_t *>(ring + (size_t)S * R * row_elems);
    uint64_t *empty = full + S;
    Real *slots = reinterpret_cast<Real *>(empty + S);                   // [nteams][2][32]
    long long r0, r1;
    row_range(p.M, p.G, g, r0, r1);
    const long long nst = (r1 - r0 + R - 1) / R;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int st = 0; st < S; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], nteams * tw);
        }
        fence_mbar_init();
    }
    __syncthreads();
    bool timed_out = false;

    if (warp == 0) {
        if (lane == 0) {
            for (long long i = 0; i < nst; ++i) {
                const int st = (int)(i % S);
                const uint32_t par = (uint32_t)((i / S) & 1);
                if (i >= S) mbar_wait_or_flag(&empty[st], par ^ 1u, timed_out);
                const long long row0 = r0 + i * R;
                const uint32_t rows = (uint32_t)min((long long)R, r1 - row0);
                mbar_arrive_expect_tx(&full[st], rows * row_bytes);
                bulk_g2s(ring + (size_t)st * R * row_elems, ws.row(s, row0), rows * row_bytes,
                         &full[st]);
            }
            // drain: the last copy into every stage has landed before the CTA can exit
            for (long long i = max(0ll, nst - S); i < nst; ++i)
                mbar_wait_or_flag(&full[i % S], (uint32_t)((i / S) & 1), timed_out);
        }
    } else {
        const int ct = threadIdx.x - 32;
        const int tthreads = 32 * tw;
        const int team = ct / tthreads, tl = ct - team * tthreads, wt = tl >> 5;
        const Real *pv = ws.vR(s, 0);
        const Real *wv = ws.w(s);
        // the operand r: in registers, except with 16 chunks per thread (the widest FP64
        // rows), where it is read through L1 for every row (it is the same for all rows)
        constexpr bool kOpL1 = VPT > 8;
        constexpr int kOpRegs = kOpL1 ? 1 : VPT;
        Chunk<Real> acc[VPT], pc[kOpRegs];
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            zero(acc[v]);
            if (!kOpL1) {
                const int c = tl + tthreads * v;
                if (c < nch) pc[v] = ldg_chunk(pv + c * E);
                else zero(pc[v]);
            }
        }
        int phase = 0;
        for (long long i = 0; i < nst; ++i) {
            const int st = (int)(i % S);
            mbar_wait_or_flag(&full[st], (uint32_t)((i / S) & 1), timed_out);
            const long long row0 = r0 + i * R;
            const int rows = (int)min((long long)R, r1 - row0);
            const Real *buf = ring + (size_t)st * R * row_elems;
            for (int rr = team; rr < rows; rr += nteams) {
                const Real *row = buf + (size_t)rr * row_elems;
                // the row's weight, loaded before the dot product so that its latency is
                // hidden behind the product and the team sum instead of following them
                const Real wrow = wv[row0 + rr];
                // narrow teams keep their chunks of the row in registers between the dot
                // product and the weighted sum (one shared-memory read of the row instead
                // of two); the 16-warp teams of the widest rows, and the 16 chunks per
                // thread of the widest FP64 rows, have no registers to spare
                constexpr bool kReread = WIDE || VPT > 8;
                constexpr int kHeld = kReread ? 1 : VPT;
                Chunk<Real> dl[kHeld];
                Real t = Real(0);
#pragma unroll
                for (int v = 0; v < VPT; ++v) {
                    const int c = tl + tthreads * v;
                    Chunk<Real> &x = dl[kReread ? 0 : v];
                    Chunk<Real> &o = pc[kOpL1 ? 0 : v];
                    if (c < nch) {
                        x = ld_chunk(row + c * E);
                        if (kOpL1) o = ldg_chunk(pv + c * E);
                    } else {
                        zero(x);
                        if (kOpL1) zero(o);
                    }
#pragma unroll
                    for (int e = 0; e < E; ++e) t += x.v[e] * o.v[e];
                }
#pragma unroll
                for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
                if (tw > 1) {
                    Real *sl = slots + (size_t)(team * 2 + phase) * 32;
                    if (lane == 0) sl[wt] = t;
                    bar_named(1 + team, tthreads);
                    t = Real(0);
                    for (int w2 = 0; w2 < tw; ++w2) t += sl[w2];
                    phase ^= 1;
                }
                const Real coef = wrow * t;
#pragma unroll
                for (int v = 0; v < VPT; ++v) {
                    const int c = tl + tthreads * v;
                    if (c < nch) {
                        if (kReread) dl[0] = ld_chunk(row + c * E);
                        const Chunk<Real> &x = dl[kReread ? 0 : v];
#pragma unroll
                        for (int e = 0; e < E; ++e) acc[v].v[e] += coef * x.v[e];
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[st]);
        }
        // team accumulators -> CTA partial (teams summed in team order via the ring)
        Real *dst = ws.part(s, g, 0);
        if (nteams == 1) {
#pragma unroll
            for (int v = 0; v < VPT; ++v) {
                const int c = tl + tthreads * v;
                if (c < nch) st_chunk(dst + c * E, acc[v]);
            }
        } else {
            bar_named(15, 32 * nteams * tw);   // every consumer is past its last ring read
#pragma unroll
            for (int v = 0; v < VPT; ++v) {
                const int c = tl + tthreads * v;
                if (c < nch) st_chunk(ring + (size_t)team * row_elems + c * E, acc[v]);
            }
            bar_named(15, 32 * nteams * tw);
            for (int c = ct; c < nch; c += 32 * nteams * tw) {
                Chunk<Real> sum = ld_chunk(ring + c * E);
                for (int t2 = 1; t2 < nteams; ++t2) {
                    const Chunk<Real> o = ld_chunk(ring + (size_t)t2 * row_elems + c * E);
#pragma unroll
                    for (int e = 0; e < E; ++e) sum.v[e] += o.v[e];
                }
                st_chunk(dst + c * E, sum);
            }
        }
    }
    if (timed_out) atomicCAS(&p.st[s].status, 0, (int)FBSDE_ERR_TIMEOUT);
}

}  // namespace dev
}  // namespace fbsde
