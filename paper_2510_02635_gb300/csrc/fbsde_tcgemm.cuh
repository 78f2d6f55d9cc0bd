// fbsde_tcgemm.cuh -- FP32-accurate matrix products on the fifth-generation tensor cores
// (tcgen05.mma, accumulator in tensor memory), for the dense contractions of the
// per-anchor solve: the distances P A^T, the moments W^T P and W^T (Y P), and per CG
// pass P V^T and T^T P.
//
// Precision: every FP32 operand value a is split as a = a_hi + a_lo, a_hi = a rounded to
// TF32 (11 significant bits), a_lo = a - a_hi (exact in FP32), and each k step issues three
// kind::tf32 MMAs into one FP32 accumulator:
//   A_hi B_hi + A_hi B_lo + A_lo B_hi.
// The dropped A_lo B_lo term (below 2^-22 |a b|) and the tensor core's truncation of the
// lo parts to TF32 (below 2^-21 |a b|) leave each product within about 1e-6 relative, the
// order of the FP32 rounding of a length-100 dot product.
//
// Tile: 128 rows (tensor-memory lanes) x 128 columns (tensor-memory columns), 16 values of
// k per pipeline stage, two stages, 256 threads.  All threads load the stage after next
// into registers and split the next one into shared memory while the tensor core runs the
// current one; one thread issues the MMAs and commits them to the stage's mbarrier, whose
// completion frees the stage.  Three blocks
// are resident per SM (64 KB of shared memory and 128 tensor-memory columns each; the
// launch bounds hold a thread to 80 registers), so one block's loads overlap another's MMAs.
// Shared memory caps an SM at three blocks, 384 of its 512 tensor-memory columns, so the
// allocation never waits for another block to free columns.
//
// Shared-memory operand layout (K-major, no swizzle): the tile of 128 rows x 16 k is four
// 16-byte chunks of k; chunk c of row r is at c * 2048 + r * 16 bytes.  In the terms of the
// tensor core's canonical layout, core matrices (8 rows x 16 bytes) are 128 bytes apart
// along the rows (stride byte offset) and 2048 bytes apart along k (leading byte offset).
#pragma once
#include "fbsde_matvec.cuh"

namespace fbsde {
namespace dev {

constexpr int kTcBM = 128, kTcBN = 128, kTcBK = 16, kTcThreads = 256, kTcStages = 2;
constexpr uint32_t kTcChunkBytes = kTcBM * 16;                  // one 16-byte k chunk of 128 rows
constexpr uint32_t kTcPartBytes = (kTcBK / 4) * kTcChunkBytes;   // one operand part: 8 KB
constexpr uint32_t kTcStageBytes = 4 * kTcPartBytes;             // A_hi, A_lo, B_hi, B_lo
constexpr uint32_t kTcSmemBytes = kTcStages * kTcStageBytes + 64;
constexpr uint32_t kTcCols = kTcBN;                               // tensor-memory columns

// Instruction descriptor of kind::tf32: FP32 accumulator (bits 4-5 = 1), A and B TF32
// (bits 7-9 and 10-12 = 2), both K-major (bits 15, 16 = 0), N / 8 at bit 17, M / 16 at bit 24.
constexpr uint32_t kTcIdesc = (1u << 4) | (2u << 7) | (2u << 10) |
                              ((uint32_t)(kTcBN >> 3) << 17) | ((uint32_t)(kTcBM >> 4) << 24);

// Shared-memory matrix descriptor: start address / 16 (bits 0-13), leading byte offset / 16
// (bits 16-29), stride byte offset / 16 (bits 32-45), descriptor version 1 (bit 46),
// no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(kTcChunkBytes >> 4) << 16) |
           ((uint64_t)(128u >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ void tc_fence_before()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Generic-proxy writes to shared memory become visible to the tensor core (async proxy).
__device__ __forceinline__ void fence_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                            uint32_t accumulate)
{
    asm volatile(
        "{\n"
        "  .reg .pred acc;\n"
        "  setp.ne.b32 acc, %4, 0;\n"
        "  tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, acc;\n"
        "}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(kTcIdesc), "r"(accumulate)
        : "memory");
}
// Arrives once on bar when every MMA this thread issued before has completed.
__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::
                     "r"(smem_u32(bar))
                 : "memory");
}
// 32 consecutive FP32 columns of this warp's 32 tensor-memory lanes (one lane per thread).
__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31}, [%32];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
          "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
          "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr)
        : "memory");
}

// a = hi + lo with hi = a rounded to 11 significant bits (magnitude rounded half up, low
// 13 bits zero) and lo = a - hi, exact.
__device__ __forceinline__ void tf32_split(float a, float &hi, float &lo)
{
    hi = __uint_as_float((__float_as_uint(a) + 0x1000u) & 0xFFFFE000u);
    lo = a - hi;
}

// Loader of one operand: each stage, a thread loads two items (tile row, 4-wide k chunk)
// of the 128-row x 16-k tile into registers, stages in increasing k order.
//   TN = false: X(row, k) = X[row * ldx + k] (k contiguous; ldx, kb and ke multiples of 4,
//               X 16-byte aligned: one 16-byte load per item).  Warp w, lane l, item u:
//               row 8 (w + 8 u) + (l & 7), chunk l >> 3, so a warp reads 8 rows x 64
//               contiguous bytes (whole sectors) and each 8-lane phase of its 16-byte
//               shared-memory stores writes 8 rows of one chunk (128 contiguous bytes).
//   TN = true:  X(row, k) = X[k * ldx + row] (rows contiguous).  Item idx = threadIdx.x +
//               256 u: row idx & 127, chunk idx >> 7, so a warp reads 32 consecutive rows of
//               one k per load.
// Rows >= nrows and k >= ke read as 0.  The item addresses are set up once and advanced by
// one stage per load; only a stage that ends past ke checks its values one by one.
template <bool TN> struct TcLoader {
    const float *p[2];   // the item's first value at the next stage's k
    uint32_t soff[2];    // the item's byte offset in an operand part
    int kq[2];           // k offset of the item within a stage (4 chunk)
    bool ok[2];          // row < nrows
    int k0, ldx;         // k of the next stage; leading dimension
    __device__ __forceinline__ TcLoader(const float *__restrict__ X, int ldx_, int row0,
                                        int nrows, int kb)
        : k0(kb), ldx(ldx_)
    {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            int row, chunk;
            if (TN) {
                const int idx = threadIdx.x + kTcThreads * u;
                row = idx & (kTcBM - 1);
                chunk = idx >> 7;
            } else {
                row = 8 * (warp + 8 * u) + (lane & 7);
                chunk = lane >> 3;
            }
            kq[u] = 4 * chunk;
            soff[u] = (uint32_t)chunk * kTcChunkBytes + (uint32_t)row * 16u;
            ok[u] = row0 + row < nrows;
            p[u] = TN ? X + (size_t)(kb + kq[u]) * ldx + (row0 + row)
                      : X + (size_t)(row0 + row) * ldx + (kb + kq[u]);
        }
    }
    __device__ __forceinline__ void load(float4 (&v)[2], int ke)
    {
        const bool full = k0 + kTcBK <= ke;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            float4 t = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            const int gk = k0 + kq[u];
            if (ok[u]) {
                if (TN) {
                    if (full || gk < ke) t.x = __ldg(p[u]);
                    if (full || gk + 1 < ke) t.y = __ldg(p[u] + ldx);
                    if (full || gk + 2 < ke) t.z = __ldg(p[u] + 2 * (size_t)ldx);
                    if (full || gk + 3 < ke) t.w = __ldg(p[u] + 3 * (size_t)ldx);
                } else if (full || gk < ke) {
                    t = __ldg(reinterpret_cast<const float4 *>(p[u]));
                }
            }
            v[u] = t;
            p[u] += TN ? (size_t)kTcBK * ldx : (size_t)kTcBK;
        }
        k0 += kTcBK;
    }
    // Split the two items into the hi and lo parts of an operand stage.
    __device__ __forceinline__ void store(const float4 (&v)[2], uint8_t *hi, uint8_t *lo) const
    {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            float4 h, l;
            tf32_split(v[u].x, h.x, l.x);
            tf32_split(v[u].y, h.y, l.y);
            tf32_split(v[u].z, h.z, l.z);
            tf32_split(v[u].w, h.w, l.w);
            *reinterpret_cast<float4 *>(hi + soff[u]) = h;
            *reinterpret_cast<float4 *>(lo + soff[u]) = l;
        }
    }
};

// Band of the batch reading (Remark 2.1): anchor m's regression uses the particles
// j = (m + q) mod M, q < Kb, so only entries (j, m) with (j - m) mod M < Kb are ever used.
// Kb >= M (or M = 0): every entry.
struct Band {
    long long M, Kb;
    // true if some j in [j0, j1) and m in [m0, m1) have (j - m) mod M < Kb
    __host__ __device__ bool hits(long long j0, long long j1, long long m0, long long m1) const
    {
        if (M <= 0 || Kb >= M) return true;
        if (j1 <= j0 || m1 <= m0) return false;
        const long long lo = j0 - (m1 - 1), hi = j1 - 1 - m0;   // offsets j - m, inclusive
        if (hi - lo + 1 >= M) return true;
        const long long lm = ((lo % M) + M) % M, hm = lm + (hi - lo);
        return lm < Kb || hm >= M;
    }
};

// Plain epilogue: C + z Mr ldc gets split z's product.
struct TcStore {
    float *C;
    int Mr, ldc;
    static constexpr bool kColSums = false, kPrefetch = false;
    struct Col {};
    struct Pre {};
    __device__ __forceinline__ Col column(int) const { return {}; }
    __device__ __forceinline__ void prefetch(int, int, const Col &, Pre &) const {}
    __device__ __forceinline__ float put(int z, int row, int col, float v, const Col &,
                                         const Pre &, int) const
    {
        C[((size_t)z * Mr + row) * ldc + col] = v;
        return 0.0f;
    }
    __device__ __forceinline__ void colsum(int, int, float) const {}
};

// Sum_k A(r, k) B(c, k) over k in [z kc, min(K, (z + 1) kc)) for split z = blockIdx.z
// (the layouts and split rule of the SIMT products:
//   TN = false: A Mr x K, B Nc x K, row-major;  TN = true: A K x Mr, B K x Nc, row-major),
// handed to the epilogue Epi element by element: Epi::column(c) once per output column,
// Epi::prefetch(r0, c, column state, pre) for the 32 rows r0.. a warp hands out next
// (issued before the accumulator is read, so its loads overlap that),
// Epi::put(z, r, c, value, column state, pre, r - r0), whose return values are summed over the rows of
// the block's 128-row tile (rows in order, 32-row quarters in order) and, with
// Epi::kColSums, passed to Epi::colsum(row tile, c, sum).
// Grid (ceil(Nc / 128), ceil(Mr / 128), splits), kTcThreads threads, kTcSmemBytes of
// dynamic shared memory.  A wait that times out sets *status = FBSDE_ERR_TIMEOUT (if 0).
// Band (batch reading): NT products (rows j, columns m) skip tiles that hold no used entry,
// writing nothing (the consumers read only entries in the band, or zero them beforehand);
// TN products (rows m, contraction over j) treat a split whose rows j miss the band of the
// tile's anchors as empty, so the epilogue writes its zero partial.
template <bool TN, class Epi>
__global__ void __launch_bounds__(kTcThreads, 3)
    k_gemm_tc(int Mr, int Nc, int K, int kc, const float *__restrict__ A, int lda,
              const float *__restrict__ B, int ldb, Epi epi, int *status, Band band)
{
    extern __shared__ __align__(1024) uint8_t tsm[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(tsm + kTcStages * kTcStageBytes);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + kTcStages);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r0 = blockIdx.y * kTcBM, c0 = blockIdx.x * kTcBN;
    const int kb = blockIdx.z * kc, ke = min(K, kb + kc);
    if (!TN && !band.hits(r0, min(Mr, r0 + kTcBM), c0, min(Nc, c0 + kTcBN))) return;
    const bool used = !TN || band.hits(kb, ke, r0, min(Mr, r0 + kTcBM));
    const int nk = (used && ke > kb) ? (ke - kb + kTcBK - 1) / kTcBK : 0;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tslot)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 32) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    bool timed_out = false;
    // Raw values of the next two stages in registers (even and odd steps): a stage's loads
    // are issued two steps before it is stored, so their latency spans two steps.
    float4 va0[2], vb0[2], va1[2], vb1[2];
    TcLoader<TN> la(A, lda, r0, Mr, kb), lb(B, ldb, c0, Nc, kb);
    if (nk > 0) {
        la.load(va0, ke);
        lb.load(vb0, ke);
    }
    if (nk > 1) {
        la.load(va1, ke);
        lb.load(vb1, ke);
    }
    auto step = [&](int t, float4 (&va)[2], float4 (&vb)[2]) {
        const int b = t & 1;
        uint8_t *stg = tsm + b * kTcStageBytes;
        // the stage's previous MMAs (step t - 2) must be done before it is overwritten
        if (t >= 2) mbar_wait_or_flag(&bar[b], (uint32_t)((t - 2) >> 1) & 1u, timed_out);
        la.store(va, stg, stg + kTcPartBytes);
        lb.store(vb, stg + 2 * kTcPartBytes, stg + 3 * kTcPartBytes);
        fence_async_smem();
        __syncthreads();
        if (t + 2 < nk) {   // loads of step t + 2 overlap this step's MMAs and the next step
            la.load(va, ke);
            lb.load(vb, ke);
        }
        if (threadIdx.x == 0) {
            tc_fence_after();
            const uint32_t ah = smem_u32(stg), al = ah + kTcPartBytes;
            const uint32_t bh = ah + 2 * kTcPartBytes, bl = ah + 3 * kTcPartBytes;
#pragma unroll
            for (int ks = 0; ks < kTcBK / 8; ++ks) {   // 8 k values = two chunks per MMA
                const uint32_t o = (uint32_t)ks * 2u * kTcChunkBytes;
                tc_mma_tf32(tmem, tc_desc(ah + o), tc_desc(bh + o), (t > 0 || ks > 0) ? 1u : 0u);
                tc_mma_tf32(tmem, tc_desc(ah + o), tc_desc(bl + o), 1u);
                tc_mma_tf32(tmem, tc_desc(al + o), tc_desc(bh + o), 1u);
            }
            tc_commit(&bar[b]);
        }
    };
    for (int t = 0; t < nk; t += 2) {
        step(t, va0, vb0);
        if (t + 1 < nk) step(t + 1, va1, vb1);
    }
    if (nk > 0) mbar_wait_or_flag(&bar[(nk - 1) & 1], (uint32_t)((nk - 1) >> 1) & 1u, timed_out);
    tc_fence_after();

    // Epilogue: warp w reads lanes 32 (w % 4) .. + 31 (rows) and columns 64 (w / 4) .. + 63,
    // 32 columns at a time, and hands them out row by row through a padded shared-memory
    // transpose (coalesced along the output rows).  The stages are free by now.
    float *scr = reinterpret_cast<float *>(tsm) + warp * (32 * 33);
    float *csm = reinterpret_cast<float *>(tsm) + 8 * (32 * 33);   // [quarter][column]
    const int q = warp & 3, h = warp >> 2;
#pragma unroll 1
    for (int cb = 0; cb < 2; ++cb) {
        const int col = 64 * h + 32 * cb;
        const int cc = c0 + col + lane;
        const typename Epi::Col cst = epi.column(cc < Nc ? cc : -1);
        typename Epi::Pre pre;
        epi.prefetch(r0 + 32 * q, cc < Nc ? cc : -1, cst, pre);
        uint32_t v[32];
        if (nk > 0) {
            tc_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)col, v);
        } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = 0u;
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) scr[lane * 33 + j] = __uint_as_float(v[j]);
        __syncwarp();
        float sum = 0.0f;
        if constexpr (Epi::kPrefetch) {   // pre is indexed by rr: unroll fully
#pragma unroll
            for (int rr = 0; rr < 32; ++rr) {
                const int row = r0 + 32 * q + rr;
                if (row < Mr && cc < Nc)
                    sum += epi.put(blockIdx.z, row, cc, scr[rr * 33 + lane], cst, pre, rr);
            }
        } else {
#pragma unroll 4
            for (int rr = 0; rr < 32; ++rr) {
                const int row = r0 + 32 * q + rr;
                if (row < Mr && cc < Nc)
                    sum += epi.put(blockIdx.z, row, cc, scr[rr * 33 + lane], cst, pre, rr);
            }
        }
        if (Epi::kColSums) csm[q * kTcBN + col + lane] = sum;
        __syncwarp();
    }
    if constexpr (Epi::kColSums) {
        __syncthreads();
        const int t = threadIdx.x;
        if (t < kTcBN && c0 + t < Nc)
            epi.colsum(blockIdx.y, c0 + t,
                       ((csm[t] + csm[kTcBN + t]) + csm[2 * kTcBN + t]) + csm[3 * kTcBN + t]);
    }
    if (timed_out && status) atomicCAS(status, 0, (int)FBSDE_ERR_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTcCols)
                     : "memory");
}

}  // namespace dev
}  // namespace fbsde
