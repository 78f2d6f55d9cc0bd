// fbsde_api.cu -- the C ABI declared in include/fbsde.h: argument checks, workspace
// layout and the launch sequence of Algorithm 1.
#include <cmath>
#include <cstring>
#include <algorithm>
#include <list>
#include <mutex>
#include <numeric>
#include <vector>

#include "fbsde_kernels.cuh"
#include "fbsde_matvec.cuh"

namespace fbsde {
namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Team geometry: a row of nch 16-byte chunks is covered by tw warps holding vpt
// chunks per thread; narrow rows use one warp per row and 8 rows per CTA.  Rows of more
// than 4096 chunks (FP64 rows beyond 8192 values) take 16 chunks per thread, so that their
// team stays within 16 warps.
bool choose_team(int nch, int &tw, int &vpt, int &teams)
{
    constexpr int vmax = 8;
    if (nch <= 32 * vmax) {
        tw = 1;
        vpt = 1;
        while (32 * vpt < nch) vpt *= 2;
    } else if (nch <= 16 * 32 * vmax) {
        vpt = vmax;
        tw = (nch + 32 * vmax - 1) / (32 * vmax);
    } else {
        vpt = 2 * vmax;
        tw = (nch + 32 * 2 * vmax - 1) / (32 * 2 * vmax);
    }
    if (32 * tw > 512) return false;
    teams = std::max(1, 256 / (32 * tw));
    return true;
}

// Check of the bounded waits: an mbarrier that nothing arrives on, waited on by every
// thread of one warp with the given limit, twice (the second wait only polls, as after
// any first timeout).  out[0] = FBSDE_ERR_TIMEOUT when every thread gave up, out[1] = the
// nanoseconds thread 0 spent.
static __global__ void __launch_bounds__(32) k_wait_probe(unsigned long long limit_ns, int *out,
                                                   unsigned long long *ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        dev::mbar_init(&bar, 1);
        dev::fence_mbar_init();
    }
    __syncwarp();
    const unsigned long long t0 = dev::globaltimer_ns();
    bool timed_out = false;
    dev::mbar_wait_or_flag(&bar, 0u, timed_out, limit_ns);
    dev::mbar_wait_or_flag(&bar, 0u, timed_out, limit_ns);
    const bool all = __all_sync(0xffffffffu, timed_out);
    if (threadIdx.x == 0) {
        *out = all ? (int)FBSDE_ERR_TIMEOUT : (int)FBSDE_OK;
        *ns = dev::globaltimer_ns() - t0;
    }
}

// check_theta: also require the device theta pointer of the kinds that read it.
int check_problem(const fbsde_problem *P, int32_t Q, bool check_theta)
{
    if (!P || Q < 1 || Q > 65535) return FBSDE_ERR_ARG;
    if (P->kind < FBSDE_AC_MANUFACTURED || P->kind > FBSDE_DRIFT_QUAD) return FBSDE_ERR_ARG;
    if (!std::isfinite(P->mu0) || !std::isfinite(P->mu1) || !std::isfinite(P->sig1))
        return FBSDE_ERR_ARG;
    if (P->kind == FBSDE_HJB_LOGQUAD && P->sig1 != 0.0) return FBSDE_ERR_ARG;
    if (P->precision != FBSDE_FP32 && P->precision != FBSDE_FP64) return FBSDE_ERR_ARG;
    if (P->d < 1 || P->d > (P->precision == FBSDE_FP64 ? FBSDE_MAX_D_FP64 : FBSDE_MAX_D))
        return FBSDE_ERR_ARG;
    if (P->N < 1 || P->M < 2 || P->M > (int64_t)1 << 31) return FBSDE_ERR_ARG;
    if (!(P->sigma > 0.0) || !std::isfinite(P->sigma)) return FBSDE_ERR_ARG;
    if (!(P->T > 0.0) || !std::isfinite(P->T)) return FBSDE_ERR_ARG;
    if (!(P->ridge_rel >= 0.0) || !std::isfinite(P->ridge_rel)) return FBSDE_ERR_ARG;
    if (!(P->cg_tol > 0.0) || P->cg_max_iter < 0 || P->newton_max_iter < 0) return FBSDE_ERR_ARG;
    if (!(P->newton_tol >= 0.0) || P->ctas < 0 || P->ctas > (1 << 20)) return FBSDE_ERR_ARG;
    if (check_theta && (P->kind == FBSDE_HJB_LOGQUAD || P->kind == FBSDE_AFFINE_TEST) &&
        !P->theta)
        return FBSDE_ERR_ARG;
    return FBSDE_OK;
}

// The scheme with Euler-Maruyama paths (a drift or a state-dependent diffusion, or a drift
// kind), rather than the driftless one whose Brownian paths are drawn by the bridge.
bool is_sde(const fbsde_problem *P)
{
    return P->mu0 != 0.0 || P->mu1 != 0.0 || P->sig1 != 0.0 || P->kind == FBSDE_DRIFT_AC ||
           P->kind == FBSDE_DRIFT_QUAD;
}

// Workspace layout; independent of every pointer in P.
int make_layout(const fbsde_problem *P, int32_t Q, Layout &L)
{
    const int st = check_problem(P, Q, false);
    if (st != FBSDE_OK) return st;
    L = Layout{};
    L.Q = Q;
    L.d = P->d;
    L.N = P->N;
    L.M = P->M;
    L.precision = P->precision;
    L.ld = (P->d + 3) / 4 * 4;
    L.real_sz = P->precision == FBSDE_FP32 ? sizeof(float) : sizeof(double);
    const int nch = (int)(L.ld * L.real_sz / 16);
    if (!choose_team(nch, L.team_warps, L.vpt, L.teams)) return FBSDE_ERR_ARG;
    L.threads = L.teams * 32 * L.team_warps;
    const long long gmax = std::max<long long>(1, P->M / kMinRowsPerCta);
    const int target = P->ctas > 0 ? P->ctas : kTargetCtas;
    L.G = (int)std::min<long long>(gmax, std::max(1, (target + Q - 1) / Q));
    // row-segment kernels: one warp per 32 * seg_vpt chunks of a row
    L.seg_vpt = nch >= 128 ? 4 : (nch >= 64 ? 2 : 1);
    L.nseg = (nch + 32 * L.seg_vpt - 1) / (32 * L.seg_vpt);
    L.row_blocks = (int)std::min<long long>(((long long)Q * P->M * L.nseg + 7) / 8,
                                            (long long)kRowBlocks);
    // per-particle kernel: 256 particles per block
    L.GP = (int)((P->M + 255) / 256);
    // matrix-free product: ring of mv_stages stages of mv_rows rows (~32 KB per stage,
    // ~200 KB of shared memory in total)
    {
        const size_t row_bytes = (size_t)L.ld * L.real_sz;
        const size_t stage_target = 32 * 1024, ring_target = 200 * 1024;
        long long R = std::max<long long>(1, (long long)(stage_target / row_bytes));
        R = std::max<long long>(L.teams, R / L.teams * L.teams);
        long long S = std::min<long long>(8, std::max<long long>(2, ring_target / (R * row_bytes)));
        // a CTA never needs a ring larger than its own rows: small instances keep their
        // ring, and so their shared memory, small (two stages of at most half their rows),
        // which lets the CTAs of concurrent instances share an SM
        const long long rows_cta = (P->M + L.G - 1) / L.G;
        if (S * R > rows_cta) {
            const long long half = ((rows_cta + 1) / 2 + L.teams - 1) / L.teams * L.teams;
            R = std::min<long long>(R, std::max<long long>(L.teams, half));
            S = std::max<long long>(2, std::min<long long>(S, (rows_cta + R - 1) / R));
        }
        L.mv_rows = (int)R;
        L.mv_stages = (int)S;
        L.mv_smem = (size_t)L.mv_stages * R * row_bytes + 2 * L.mv_stages * sizeof(uint64_t) +
                    (size_t)L.teams * 2 * 32 * L.real_sz;
        if (L.mv_smem > 227 * 1024) return FBSDE_ERR_ARG;
    }
    // fused per-level step (FP32 rows up to kStepMaxLd floats): R rows per stage, the
    // largest of {1, 3, 5, 15, 30} with R ld <= kStepElems (at most 30: one service-warp lane
    // per row), T = 480 / R threads per row in the row pass (whole warps, or half-warps at
    // R = 30), VM = ceil(nch / T) chunks per thread; column pass in row groups of
    // tpr = min(480, nch) threads; a two-slot ring of stages in shared memory
    L.sde = is_sde(P) ? 1 : 0;
    L.fused = !L.sde && P->precision == FBSDE_FP32 && L.ld <= kStepMaxLd;
    if (L.fused) {
        constexpr int kRows[5] = {1, 3, 5, 15, 30};
        int R = 1;
        for (int r : kRows)
            if ((size_t)r * L.ld <= (size_t)kStepElems) R = r;
        L.st_R = R;
        L.st_T = 480 / R;
        L.st_vm1 = (nch + L.st_T - 1) / L.st_T;
        L.st_tpr = std::min(480, nch);
        L.st_RG = 480 / L.st_tpr;
        L.st_vm3 = (nch + L.st_tpr - 1) / L.st_tpr;
        L.st_vm = L.st_vm1;
        L.st_nslot = 2;
        const size_t ring = (size_t)2 * R * L.ld;
        const size_t red = L.st_RG > 1 ? (size_t)L.st_RG * 3 * nch * 4 : 0;
        L.st_region = std::max(ring, red);
        const size_t tail = L.st_vm3 > 5 ? (size_t)3 * (nch - 5 * 480) * 16 : 0;
        L.st_smem = (3 * (size_t)L.ld + L.st_region) * sizeof(float) + 4 * 32 * 16 + 48 + tail;
        if (L.st_vm > 6 || L.st_vm3 > L.st_vm || (L.st_vm3 > 5 && R != 1) ||
            L.st_smem > 227 * 1024)
            return FBSDE_ERR_ARG;
    }
    // CTAs per query of the fused step (one CTA per SM): whole waves of 152 CTAs where
    // possible, at least four stages per CTA; 4..1 waves first, then 5..8
    L.Gs = L.G;
    if (L.fused) {
        const long long gmax_s = std::max<long long>(1, P->M / (4LL * L.st_R));
        double best = -1.0;
        for (int W : {4, 3, 2, 1, 5, 6, 7, 8}) {
            const long long g = std::min<long long>(gmax_s, (152LL * W + Q - 1) / Q);
            const double waves = (double)(g * Q) / 152.0;
            const double eff = waves / std::ceil(waves);
            if (eff > best + 1e-9) {
                best = eff;
                L.Gs = (int)g;
            }
            if (eff >= 0.99) break;
        }
    }
    L.GS = std::max(L.GP, L.fused ? L.Gs : 0);
    // partial reduction: tiles of kRedTile elements, red_groups warps per tile, each adding
    // about four of the G partials
    L.nblk = (L.ld + kRedTile - 1) / kRedTile;
    L.red_groups = std::min(16, std::max(4, (L.G + 3) / 4));
    // moments: column tiles of 256 * mom_vm chunks
    L.mom_vm = nch > 256 ? 2 : 1;
    L.mom_tiles = (nch + 256 * L.mom_vm - 1) / (256 * L.mom_vm);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, kAlign);
        return o;
    };
    const size_t Qs = (size_t)Q, Ms = (size_t)P->M, lds = (size_t)L.ld;
    L.off_delta = take(Qs * Ms * lds * L.real_sz);
    L.off_Y = take(Qs * Ms * sizeof(double));
    L.off_w = take(Qs * Ms * L.real_sz);
    L.off_coef = take(Qs * Ms * 3 * L.real_sz);
    L.off_segp = take(Qs * Ms * (size_t)L.nseg * kSegSums * L.real_sz);
    L.off_part = take(Qs * std::max(L.G, L.Gs) * kPartVecs * lds * L.real_sz);
    L.off_spart = take(Qs * L.GS * kPartScal * sizeof(double));
    L.off_vec64 = take(Qs * kVec64 * lds * sizeof(double));
    L.off_vecR = take((Qs * kVecR + 1) * lds * L.real_sz);
    L.off_state = take(Qs * sizeof(SolveState));
    L.off_bpart = take(Qs * (size_t)L.nblk * kBpart * sizeof(double));
    if (L.sde) {
        // Euler-Maruyama rows: checkpoints at the levels s, 2s, .. below N and one segment of
        // s - 1 levels, s = ceil(sqrt N): about 2 sqrt(N) slabs of Q M ld instead of N - 1,
        // for one more forward step per level on the way back
        int sq = 1;
        while (sq * sq < P->N) ++sq;
        L.sde_s = sq;
        L.sde_ncp = (P->N - 1) / sq;
        L.sde_slots = L.sde_ncp + sq - 1;
        L.off_store = take((size_t)L.sde_slots * Qs * Ms * lds * L.real_sz);
        L.off_anchor = take(Qs * (size_t)(P->N + 1) * lds * L.real_sz);
    }
    L.total = off;
    // reverse sweep: tape of the primal plus three adjoint vectors per query
    L.off_tape_w = take((size_t)P->N * Qs * Ms * L.real_sz);
    L.off_tape_Y = take((size_t)(P->N + 1) * Qs * Ms * sizeof(double));
    L.off_tape_v = take(Qs * (size_t)P->N * 2 * lds * sizeof(double));
    L.off_tape_s = take(Qs * (size_t)P->N * 4 * sizeof(double));
    L.off_adj_v = take(Qs * 3 * lds * sizeof(double));
    L.total_adjoint = off;
    return FBSDE_OK;
}

Params make_params(const fbsde_problem *P, const Layout &L, void *ws, uint64_t seed,
                   uint32_t solve0, double *u0, double *grad, const fbsde_trace *tr)
{
    Params p{};
    p.kind = P->kind;
    p.d = P->d;
    p.ld = L.ld;
    p.N = P->N;
    p.G = L.G;
    p.Q = L.Q;
    p.nseg = L.nseg;
    p.GP = L.GP;
    p.GS = L.GS;
    p.nsp = L.fused ? L.Gs : L.GP;
    p.st_R = L.st_R;
    p.st_T = L.st_T;
    p.st_vm1 = L.st_vm1;
    p.st_tpr = L.st_tpr;
    p.st_RG = L.st_RG;
    p.st_vm3 = L.st_vm3;
    p.st_nslot = L.st_nslot;
    p.st_region = (long long)L.st_region;
    p.mv_rows = L.mv_rows;
    p.mv_stages = L.mv_stages;
    p.team_warps = L.team_warps;
    p.M = P->M;
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
    p.walk = -1;
    p.theta = P->theta;
    p.key0 = (uint32_t)seed;
    p.key1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {   // Weyl sequence of the Philox key, one entry per round
        p.rk0[r] = p.key0 + (uint32_t)r * 0x9E3779B9u;
        p.rk1[r] = p.key1 + (uint32_t)r * 0xBB67AE85u;
    }
    p.solve0 = solve0;
    p.sde = L.sde;
    p.mu0 = P->mu0;
    p.mu1 = P->mu1;
    p.sig1 = P->sig1;
    char *base = static_cast<char *>(ws);
    p.anchor = L.sde ? base + L.off_anchor : nullptr;
    p.delta = base + L.off_delta;
    p.Y = reinterpret_cast<double *>(base + L.off_Y);
    p.w = base + L.off_w;
    p.coef = base + L.off_coef;
    p.segp = base + L.off_segp;
    p.part = base + L.off_part;
    p.spart = reinterpret_cast<double *>(base + L.off_spart);
    p.vec64 = reinterpret_cast<double *>(base + L.off_vec64);
    p.vecR = base + L.off_vecR;
    p.st = reinterpret_cast<SolveState *>(base + L.off_state);
    p.bpart = reinterpret_cast<double *>(base + L.off_bpart);
    p.nblk = L.nblk;
    p.u0 = u0;
    p.grad = grad;
    if (tr) {
        p.tr_alpha = tr->alpha;
        p.tr_alpha_x = tr->alpha_x;
        p.tr_cg = tr->cg_iters;
        p.tr_newton = tr->newton_iters;
        p.tr_x_N = tr->x_N;
        p.tr_y_N = tr->y_N;
    }
    return p;
}

// ---------------------------------------------------------------------------
// Launch profiler: counts launches per kernel family and brackets the first `cap`
// launches with CUDA events on the launching stream.
// ---------------------------------------------------------------------------
struct Profiler {
    std::mutex mu;
    bool on = false;
    int cap = 0, used = 0;
    uint32_t mask = (1u << FBSDE_NUM_KERNELS) - 1;
    std::vector<cudaEvent_t> ev;
    std::vector<int> fam;
    int64_t launches[FBSDE_NUM_KERNELS] = {};
};
Profiler g_prof;

struct ProfScope {
    int slot = -1;
    cudaStream_t s;
    ProfScope(int family, cudaStream_t st) : s(st)
    {
        if (!g_prof.on || family < 0) return;
        std::lock_guard<std::mutex> lk(g_prof.mu);
        g_prof.launches[family] += 1;
        if (((g_prof.mask >> family) & 1u) && g_prof.used < g_prof.cap) {
            slot = g_prof.used++;
            g_prof.fam[slot] = family;
            cudaEventRecord(g_prof.ev[2 * slot], s);
        }
    }
    ~ProfScope()
    {
        if (slot >= 0) cudaEventRecord(g_prof.ev[2 * slot + 1], s);
    }
};

// True while the launch profiler brackets product launches with events.
bool profiling_products()
{
    std::lock_guard<std::mutex> lk(g_prof.mu);
    return g_prof.on && ((g_prof.mask >> FBSDE_K_MATVEC) & 1u);
}

// Where the launches go: eagerly on a stream (with the optional launch profiler), or
// into a CUDA graph being captured on that stream, with each CG loop as a conditional
// while node whose body is captured on a second stream.  graph_tail (eager only): the
// CG passes that the eager loop does not launch one by one run as a cached CUDA graph.
struct Rec {
    cudaStream_t s;
    bool capture;
    cudaStream_t body;
    bool graph_tail;
};

#define FBSDE_TRY(fam, call)                                                                 \
    do {                                                                                     \
        ProfScope ps_(r.capture ? -1 : (fam), r.s);                                          \
        if ((e = (call)) != cudaSuccess) return e;                                           \
    } while (0)

constexpr int kCgUnroll = 2;   // CG passes per iteration of the conditional while node

// The CG loop captured into the graph being built on stream s: a reset kernel that sets
// the loop condition, then a conditional while node whose body (product, reduction, CG
// update) is captured on the stream `body`; k_cg_update keeps the condition at 1 while
// some query iterates and fewer than cg_max_iter passes ran.
template <typename Real>
cudaError_t cg_capture(const Params &p, const Layout &L, cudaStream_t s, cudaStream_t b)
{
    using LR = Launch<Real>;
    cudaError_t e;
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *ed = nullptr;
    size_t nd = 0;
    if ((e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, &ed, &nd)) != cudaSuccess) return e;
    if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
    cudaGraphConditionalHandle h;
    if ((e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault)) != cudaSuccess)
        return e;
    if ((e = LR::cg_reset(p, h, s)) != cudaSuccess) return e;
    if ((e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, &ed, &nd)) != cudaSuccess) return e;
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if ((e = cudaGraphAddNode(&node, g, deps, ed, nd, &np)) != cudaSuccess) return e;
    if ((e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1,
                                                 cudaStreamSetCaptureDependencies)) != cudaSuccess)
        return e;
    cudaGraph_t body = np.conditional.phGraph_out[0];
    if ((e = cudaStreamBeginCaptureToGraph(b, body, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeRelaxed)) != cudaSuccess)
        return e;
    // kCgUnroll passes per iteration of the while node: each iteration of a conditional
    // node costs a device-side launch of its body graph; passes after convergence exit at
    // once (the kernels test the query's done flag), and every pass updates the condition
    cudaError_t eb = cudaSuccess;
    for (int u = 0; u < kCgUnroll && eb == cudaSuccess; ++u) {
        eb = LR::matvec(p, L, b);
        if (eb == cudaSuccess) eb = LR::reduce(p, L, 1, 5, 1, b);
        if (eb == cudaSuccess) eb = LR::cg_update(p, L, h, 1, b);
    }
    cudaGraph_t ended = nullptr;
    e = cudaStreamEndCapture(b, &ended);
    return eb != cudaSuccess ? eb : e;
}

// Cache of instantiated CG-loop graphs for the eager entry points, keyed by device,
// precision and the bytes of the layout and of the parameters the CG kernels see (the
// level-dependent fields are zeroed: the product, reduction and update kernels do not
// read them, so every level of a solve shares one graph).  Least-recently used entries
// beyond kCgCacheSize are destroyed after their last launch completes.  The cache is
// never freed, so no CUDA call runs from a static destructor at process exit.
constexpr size_t kCgCacheSize = 32;
constexpr int kEagerPasses = FBSDE_PROFILED_EAGER_PASSES;

struct CgGraph {
    int dev;
    std::vector<unsigned char> key;
    cudaGraphExec_t exec;
    cudaEvent_t last;
};
struct CgCache {
    std::mutex mu;
    std::list<CgGraph> lru;
    cudaStream_t cap[64] = {}, body[64] = {};
};
CgCache *g_cg = new CgCache();

template <typename Real> cudaError_t cg_graph_launch(const Params &p, const Layout &L, cudaStream_t s)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    Params q;
    std::memset(&q, 0, sizeof q);
    q = p;
    q.level = 0;
    q.newton_level = 0;
    q.walk = 0;
    q.wa = q.wb = 0.0;
    std::vector<unsigned char> key(sizeof q + sizeof L + 1);
    std::memcpy(key.data(), &q, sizeof q);
    std::memcpy(key.data() + sizeof q, &L, sizeof L);
    key[sizeof q + sizeof L] = (unsigned char)sizeof(Real);
    std::lock_guard<std::mutex> lk(g_cg->mu);
    auto it = g_cg->lru.begin();
    for (; it != g_cg->lru.end(); ++it)
        if (it->dev == dev && it->key == key) break;
    if (it == g_cg->lru.end()) {
        if (!g_cg->cap[dev]) {
            if ((e = cudaStreamCreateWithFlags(&g_cg->cap[dev], cudaStreamNonBlocking)) != cudaSuccess)
                return e;
            if ((e = cudaStreamCreateWithFlags(&g_cg->body[dev], cudaStreamNonBlocking)) != cudaSuccess)
                return e;
        }
        if ((e = cudaStreamBeginCapture(g_cg->cap[dev], cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return e;
        const cudaError_t ec = cg_capture<Real>(q, L, g_cg->cap[dev], g_cg->body[dev]);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(g_cg->cap[dev], &g);
        if (ec != cudaSuccess || e != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            return ec != cudaSuccess ? ec : (e != cudaSuccess ? e : cudaErrorUnknown);
        }
        CgGraph c{dev, key, nullptr, nullptr};
        e = cudaGraphInstantiate(&c.exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&c.last, cudaEventDisableTiming)) != cudaSuccess) {
            cudaGraphExecDestroy(c.exec);
            return e;
        }
        g_cg->lru.push_front(c);
        while (g_cg->lru.size() > kCgCacheSize) {
            CgGraph &old = g_cg->lru.back();
            cudaEventSynchronize(old.last);
            cudaGraphExecDestroy(old.exec);
            cudaEventDestroy(old.last);
            g_cg->lru.pop_back();
        }
        it = g_cg->lru.begin();
    } else if (it != g_cg->lru.begin()) {
        g_cg->lru.splice(g_cg->lru.begin(), g_cg->lru, it);
        it = g_cg->lru.begin();
    }
    if ((e = cudaGraphLaunch(it->exec, s)) != cudaSuccess) return e;
    return cudaEventRecord(it->last, s);
}

// The CG iterations of one regression (all queries of the launch together).  Eager: the
// passes are launched one by one (kernels of queries that have converged exit at once),
// or, with graph_tail, handed to a cached CUDA graph whose conditional while loop runs
// only the passes some query needs.  While the launch profiler times the product kernel,
// the first kEagerPasses passes stay eager so their products can be bracketed by events.
// A stream that is itself being captured gets the eager passes.
template <typename Real> cudaError_t cg_loop(const Params &p, const Layout &L, const Rec &r)
{
    using LR = Launch<Real>;
    cudaError_t e;
    const cudaStream_t s = r.s;
    if (r.capture) return cg_capture<Real>(p, L, s, r.body);
    bool tail = r.graph_tail;
    if (tail) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if ((e = cudaStreamIsCapturing(s, &cs)) != cudaSuccess) return e;
        tail = cs == cudaStreamCaptureStatusNone;
    }
    const int eager = !tail ? p.cg_max_iter
                            : (profiling_products() ? std::min(p.cg_max_iter, kEagerPasses) : 0);
    for (int it = 0; it < eager; ++it) {
        FBSDE_TRY(FBSDE_K_MATVEC, LR::matvec(p, L, s));
        FBSDE_TRY(FBSDE_K_REDUCE, LR::reduce(p, L, 1, 5, 1, s));
        FBSDE_TRY(FBSDE_K_CG_STEP, LR::cg_update(p, L, 0, 0, s));
    }
    if (eager < p.cg_max_iter) return cg_graph_launch<Real>(p, L, s);
    return cudaSuccess;
}

template <typename Real>
cudaError_t run_sde(Params p, const Layout &L, const double *x0, const double *theta, const Rec &r);

// Algorithm 1: forward sweep, then the backward levels k = N-1..0.  Each level: the CG
// solve of its regression (moments already reduced), then, for k >= 1, the particle
// update to level k and the moments of the level k-1 regression.
template <typename Real>
cudaError_t run(Params p, const Layout &L, const double *x0, const double *theta, const Rec &r)
{
    if (L.sde) return run_sde<Real>(p, L, x0, theta, r);
    using LR = Launch<Real>;
    cudaError_t e;
    const cudaStream_t s = r.s;
    FBSDE_TRY(FBSDE_K_SETUP, LR::setup(p, x0, theta, s));
    // the fused step tiles the rows over L.Gs CTAs per query: its partial vectors are
    // reduced with that count (the products keep L.G)
    Params ps = p;
    ps.G = L.Gs;
    ps.level = p.N;
    p.level = p.N;
    if (L.fused) {   // forward sweep end point, g and the first regression's moments in one pass
        FBSDE_TRY(FBSDE_K_STEP, LR::step(ps, L, s));
    } else {
        FBSDE_TRY(FBSDE_K_FORWARD, LR::forward(p, L, s));
        FBSDE_TRY(FBSDE_K_PARTICLES, LR::particles(p, L, s));
    }
    if (p.tr_x_N || p.tr_y_N) FBSDE_TRY(FBSDE_K_TRACE, LR::trace_forward(p, L, s));
    if (!L.fused) FBSDE_TRY(FBSDE_K_MOMENTS, LR::moments(p, L, s));
    FBSDE_TRY(FBSDE_K_REDUCE, LR::reduce(ps, L, 3, 3, 0, s));
    p.newton_level = -1;
    FBSDE_TRY(FBSDE_K_FINALIZE, LR::moments_finalize(p, L, 0, s));
    for (int k = p.N - 1; k >= 0; --k) {
        p.level = k;
        if ((e = cg_loop<Real>(p, L, r)) != cudaSuccess) return e;
        FBSDE_TRY(FBSDE_K_CG_POST, LR::cg_post(p, L, s));
        if (k >= 1) {
            if (L.fused) {   // the whole level step in one pass over the rows
                ps = p;
                ps.G = L.Gs;
                FBSDE_TRY(FBSDE_K_STEP, LR::step(ps, L, s));
                FBSDE_TRY(FBSDE_K_REDUCE, LR::reduce(ps, L, 3, 3, 0, s));
            } else {
                FBSDE_TRY(FBSDE_K_UPDATE, LR::update(p, L, s));
                FBSDE_TRY(FBSDE_K_PARTICLES, LR::particles(p, L, s));
                FBSDE_TRY(FBSDE_K_MOMENTS, LR::moments(p, L, s));
                FBSDE_TRY(FBSDE_K_REDUCE, LR::reduce(p, L, 3, 3, 0, s));
            }
            p.newton_level = k;
            FBSDE_TRY(FBSDE_K_FINALIZE, LR::moments_finalize(p, L, 1, s));
        }
    }
    return cudaSuccess;
}

// Algorithm 1 with Euler-Maruyama paths (2.7).  The forward sweep keeps the rows of the
// levels s, 2s, .. (checkpoints) and of the last segment; on the way back the level-k rows
// come from a checkpoint or the segment buffer (a segment is recomputed from its checkpoint
// when the sweep enters it) and are copied into the row buffer by the row-sum kernel, so
// every level's kernels (and the cached CG-loop graph) see the same rows pointer.  Per level k: row sums
// (k_sde_rows), the kernel scale (k_sde_rho), the per-particle values and weights, the
// moments and the regression set-up of level k - 1.
template <typename Real>
cudaError_t run_sde(Params p, const Layout &L, const double *x0, const double *theta, const Rec &r)
{
    using LR = Launch<Real>;
    cudaError_t e;
    const cudaStream_t s = r.s;
    const int N = p.N, sq = L.sde_s;
    const size_t slab = (size_t)L.Q * (size_t)L.M * L.ld * L.real_sz;
    char *store = static_cast<char *>(p.delta) - L.off_delta + L.off_store;
    // slot of a stored level 1 <= l < N: checkpoint l / sq - 1, or segment slot l % sq - 1
    auto slot = [&](int l) -> void * {
        const int i = l % sq == 0 ? l / sq - 1 : L.sde_ncp + l % sq - 1;
        return store + (size_t)i * slab;
    };
    FBSDE_TRY(FBSDE_K_SETUP, LR::setup(p, x0, theta, s));
    FBSDE_TRY(FBSDE_K_SETUP, LR::sde_anchor(p, L, s));
    const void *from = nullptr;
    for (int k = 0; k < N; ++k) {
        void *to = k + 1 == N ? p.delta : slot(k + 1);
        FBSDE_TRY(FBSDE_K_FORWARD, LR::sde_forward(p, L, k, from, to, s));
        from = to;
    }
    int seg = (N - 1) / sq * sq;   // the segment whose levels the forward sweep left in place
    p.level = N;
    p.newton_level = -1;
    FBSDE_TRY(FBSDE_K_UPDATE, LR::sde_rows(p, L, N, nullptr, s));
    FBSDE_TRY(FBSDE_K_PARTICLES, LR::sde_rho(p, L, s));
    FBSDE_TRY(FBSDE_K_PARTICLES, LR::particles(p, L, s));
    if (p.tr_x_N || p.tr_y_N) FBSDE_TRY(FBSDE_K_TRACE, LR::trace_forward(p, L, s));
    FBSDE_TRY(FBSDE_K_MOMENTS, LR::moments(p, L, s));
    FBSDE_TRY(FBSDE_K_REDUCE, LR::reduce(p, L, 3, 3, 0, s));
    FBSDE_TRY(FBSDE_K_FINALIZE, LR::moments_finalize(p, L, 0, s));
    for (int k = N - 1; k >= 0; --k) {
        p.level = k;
        if ((e = cg_loop<Real>(p, L, r)) != cudaSuccess) return e;
        FBSDE_TRY(FBSDE_K_CG_POST, LR::cg_post(p, L, s));
        if (k == 0) break;
        const int b = k / sq * sq;
        if (b != k && b != seg) {   // recompute the segment b+1 .. min(b+sq-1, N-1)
            const void *src = b == 0 ? nullptr : slot(b);
            for (int l = b + 1; l < std::min(b + sq, N); ++l) {
                FBSDE_TRY(FBSDE_K_FORWARD, LR::sde_forward(p, L, l - 1, src, slot(l), s));
                src = slot(l);
            }
            seg = b;
        }
        // the level's rows from their slot into the row buffer, with the row sums
        FBSDE_TRY(FBSDE_K_UPDATE, LR::sde_rows(p, L, k, slot(k), s));
        FBSDE_TRY(FBSDE_K_PARTICLES, LR::sde_rho(p, L, s));
        FBSDE_TRY(FBSDE_K_PARTICLES, LR::particles(p, L, s));
        FBSDE_TRY(FBSDE_K_MOMENTS, LR::moments(p, L, s));
        FBSDE_TRY(FBSDE_K_REDUCE, LR::reduce(p, L, 3, 3, 0, s));
        p.newton_level = k;
        FBSDE_TRY(FBSDE_K_FINALIZE, LR::moments_finalize(p, L, 1, s));
    }
    return cudaSuccess;
}

// Reverse sweep (see fbsde_adjoint.cuh): the primal is re-run with its tape recorded,
// then for k = 0..N-1 the adjoint solve of level k, the per-particle adjoint and the
// column sums, walking the particle rows up from Delta_1 by inverting the Brownian-bridge
// steps with the regenerated normals.
template <typename Real>
cudaError_t run_adjoint(Params p, const Layout &L, const double *x0, const double *theta,
                        const double *ubar, double *x0bar, double *thetabar, char *base,
                        const Rec &r)
{
    using LR = Launch<Real>;
    cudaError_t e;
    const cudaStream_t s = r.s;
    p.tape_w = base + L.off_tape_w;
    p.tape_Y = reinterpret_cast<double *>(base + L.off_tape_Y);
    p.tape_v = reinterpret_cast<double *>(base + L.off_tape_v);
    p.tape_s = reinterpret_cast<double *>(base + L.off_tape_s);
    p.adj_v = reinterpret_cast<double *>(base + L.off_adj_v);
    if ((e = run<Real>(p, L, x0, theta, r)) != cudaSuccess) return e;
    FBSDE_TRY(FBSDE_K_ADJOINT, LR::adj_init(p, L, ubar, s));
    int mode_b = 0, mode_c = 0;  // terminal column functions per kind
    switch (p.kind) {
    case FBSDE_AC_MANUFACTURED:
    case FBSDE_COS_LINEAR_TEST: mode_b = 1; break;
    case FBSDE_HJB_LOGQUAD: mode_b = 2; mode_c = 1; break;
    case FBSDE_AFFINE_TEST: mode_c = 2; break;
    case FBSDE_AC_DOUBLEWELL: mode_b = 2; break;
    }
    for (int k = 0; k < p.N; ++k) {
        p.level = k;
        // weights of level k into the weight buffer (every level's kernels, and so the
        // cached CG-loop graph, then see the same pointer)
        {
            const size_t wb = (size_t)L.Q * L.M * sizeof(Real);
            if ((e = cudaMemcpyAsync(p.w, static_cast<const char *>(p.tape_w) + (size_t)k * wb, wb,
                                     cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
                return e;
        }
        if (k >= 1) {   // start from the previous level's solution: one product
            FBSDE_TRY(FBSDE_K_ADJOINT, LR::adj_warm(p, L, s));
            FBSDE_TRY(FBSDE_K_MATVEC, LR::matvec(p, L, s));
            FBSDE_TRY(FBSDE_K_REDUCE, LR::reduce(p, L, 1, 5, 0, s));
        }
        FBSDE_TRY(FBSDE_K_ADJOINT, LR::adj_setup(p, L, k >= 1 ? 1 : 0, s));
        if ((e = cg_loop<Real>(p, L, r)) != cudaSuccess) return e;
        FBSDE_TRY(FBSDE_K_ADJOINT, LR::adj_post(p, L, s));
        FBSDE_TRY(FBSDE_K_ADJOINT, LR::adj_rows(p, L, s));
        FBSDE_TRY(FBSDE_K_ADJOINT, LR::adj_zlevel(p, L, s));
        FBSDE_TRY(FBSDE_K_ADJOINT, LR::adj_particles(p, L, s));
        const bool terminal = k + 1 == p.N;
        const int mb = terminal ? mode_b : (p.kind == FBSDE_AC_MANUFACTURED ? 1 : 0);
        FBSDE_TRY(FBSDE_K_ADJOINT, LR::adj_colsum(p, L, mb, terminal ? mode_c : 0, s));
        FBSDE_TRY(FBSDE_K_REDUCE, LR::reduce(p, L, 3, 3, 0, s));
        FBSDE_TRY(FBSDE_K_ADJOINT, LR::adj_finalize(p, L, s));
        if (!terminal) {  // rows Delta_{k+1} -> Delta_{k+2}: the bridge step of level k+1 inverted
            Params q = p;
            q.level = k + 1;
            q.walk = +1;
            FBSDE_TRY(FBSDE_K_UPDATE, LR::update(q, L, s));
        }
    }
    FBSDE_TRY(FBSDE_K_ADJOINT, LR::adj_output(p, L, x0bar, thetabar, s));
    return cudaSuccess;
}

#undef FBSDE_TRY

int solve_impl(const fbsde_problem *P, int32_t Q, const double *x0, const double *theta,
               uint64_t seed, uint32_t solve_index0, double *u0, double *grad_u0,
               const fbsde_trace *trace, void *workspace, size_t workspace_bytes,
               cudaStream_t stream, bool graph_tail = true)
{
    Layout L;
    int st = check_problem(P, Q, false);
    if (st != FBSDE_OK) return st;
    if ((P->kind == FBSDE_HJB_LOGQUAD || P->kind == FBSDE_AFFINE_TEST) && !theta)
        return FBSDE_ERR_ARG;
    st = make_layout(P, Q, L);
    if (st != FBSDE_OK) return st;
    if (!x0 || !u0) return FBSDE_ERR_ARG;
    if (!workspace || workspace_bytes < L.total || (reinterpret_cast<uintptr_t>(workspace) % kAlign))
        return FBSDE_ERR_WORKSPACE;
    const Params p = make_params(P, L, workspace, seed, solve_index0, u0, grad_u0, trace);
    const Rec r{stream, false, nullptr, graph_tail};
    const cudaError_t e = P->precision == FBSDE_FP32 ? run<float>(p, L, x0, theta, r)
                                                     : run<double>(p, L, x0, theta, r);
    return e == cudaSuccess ? FBSDE_OK : FBSDE_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Plans.
// ---------------------------------------------------------------------------
struct PlanInstance {
    fbsde_instance in;
    Layout L;
    size_t offset;
};

int plan_layout(int32_t n, const fbsde_instance *inst, std::vector<PlanInstance> &out, size_t &total)
{
    if (n < 1 || !inst) return FBSDE_ERR_ARG;
    out.clear();
    total = 0;
    for (int i = 0; i < n; ++i) {
        PlanInstance pi;
        pi.in = inst[i];
        int st = check_problem(&pi.in.problem, pi.in.Q, true);
        if (st != FBSDE_OK) return st;
        if ((st = make_layout(&pi.in.problem, pi.in.Q, pi.L)) != FBSDE_OK) return st;
        if (!pi.in.x0 || !pi.in.u0) return FBSDE_ERR_ARG;
        pi.offset = total;
        total = align_up(total + pi.L.total, kAlign);
        out.push_back(pi);
    }
    return FBSDE_OK;
}

__global__ void k_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
        const uint4 o = dev::philox4x32_10(c, key[0], key[1]);
        out[4 * i] = o.x;
        out[4 * i + 1] = o.y;
        out[4 * i + 2] = o.z;
        out[4 * i + 3] = o.w;
    }
}

}  // namespace
}  // namespace fbsde

namespace fbsde {
// fbsde_solve with every CG pass launched on the stream (no CUDA graph is created,
// instantiated or cached), for the entry point that must allocate nothing.
int solve_launches_only(const fbsde_problem *P, int32_t Q, const double *x0, uint64_t seed,
                        uint32_t solve_index0, double *u0, double *grad_u0, void *workspace,
                        size_t workspace_bytes, cudaStream_t stream)
{
    return solve_impl(P, Q, x0, P ? P->theta : nullptr, seed, solve_index0, u0, grad_u0,
                      nullptr, workspace, workspace_bytes, stream, false);
}
}  // namespace fbsde

using namespace fbsde;

struct fbsde_plan {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaStream_t> streams;   // capture origin, loop bodies, branches
    std::vector<cudaEvent_t> events;
    std::vector<PlanInstance> inst;
    void *workspace = nullptr;
};

static void plan_free(fbsde_plan *pl)
{
    if (!pl) return;
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    for (cudaEvent_t e : pl->events) cudaEventDestroy(e);
    for (cudaStream_t s : pl->streams) cudaStreamDestroy(s);
    delete pl;
}

extern "C" {

size_t fbsde_workspace_bytes(const fbsde_problem *P, int32_t Q)
{
    Layout L;
    return make_layout(P, Q, L) == FBSDE_OK ? L.total : 0;
}

int fbsde_solve(const fbsde_problem *P, int32_t Q, const double *x0, uint64_t seed,
                uint32_t solve_index0, double *u0, double *grad_u0, const fbsde_trace *trace,
                void *workspace, size_t workspace_bytes, fbsde_stream_t stream)
{
    return solve_impl(P, Q, x0, P ? P->theta : nullptr, seed, solve_index0, u0, grad_u0, trace,
                      workspace, workspace_bytes, reinterpret_cast<cudaStream_t>(stream));
}

size_t fbsde_adjoint_workspace_bytes(const fbsde_problem *P, int32_t Q)
{
    Layout L;
    return make_layout(P, Q, L) == FBSDE_OK ? L.total_adjoint : 0;
}

int fbsde_adjoint(const fbsde_problem *P, int32_t Q, const double *x0, uint64_t seed,
                  uint32_t solve_index0, const double *u0_bar, double *u0, double *grad_u0,
                  double *x0_bar, double *theta_bar, void *workspace, size_t workspace_bytes,
                  fbsde_stream_t stream)
{
    Layout L;
    int st = check_problem(P, Q, true);
    if (st != FBSDE_OK) return st;
    if (is_sde(P)) return FBSDE_ERR_ARG;   // the reverse sweep walks the Brownian bridge
    st = make_layout(P, Q, L);
    if (st != FBSDE_OK) return st;
    if (!x0 || !u0_bar || !u0 || !x0_bar) return FBSDE_ERR_ARG;
    if (theta_bar && !(P->kind == FBSDE_HJB_LOGQUAD || P->kind == FBSDE_AFFINE_TEST))
        return FBSDE_ERR_ARG;
    if (!workspace || workspace_bytes < L.total_adjoint ||
        (reinterpret_cast<uintptr_t>(workspace) % kAlign))
        return FBSDE_ERR_WORKSPACE;
    const Params p = make_params(P, L, workspace, seed, solve_index0, u0, grad_u0, nullptr);
    const Rec r{reinterpret_cast<cudaStream_t>(stream), false, nullptr, true};
    char *base = static_cast<char *>(workspace);
    const cudaError_t e =
        P->precision == FBSDE_FP32
            ? run_adjoint<float>(p, L, x0, P->theta, u0_bar, x0_bar, theta_bar, base, r)
            : run_adjoint<double>(p, L, x0, P->theta, u0_bar, x0_bar, theta_bar, base, r);
    return e == cudaSuccess ? FBSDE_OK : FBSDE_ERR_CUDA;
}

size_t fbsde_host_staging_bytes(const fbsde_problem *P, int32_t Q)
{
    if (check_problem(P, Q, false) != FBSDE_OK) return 0;
    const size_t Qs = (size_t)Q, ds = (size_t)P->d;
    return align_up(Qs * ds * 8, kAlign) * 2 + align_up(Qs * 8, kAlign) + align_up(ds * 8, kAlign);
}

int fbsde_solve_host(const fbsde_problem *P, int32_t Q, const double *x0_host, uint64_t seed,
                     uint32_t solve_index0, double *u0_host, double *grad_u0_host,
                     void *workspace, size_t workspace_bytes, fbsde_stream_t stream)
{
    if (!P || !x0_host || !u0_host) return FBSDE_ERR_ARG;
    const bool needs_theta = P->kind == FBSDE_HJB_LOGQUAD || P->kind == FBSDE_AFFINE_TEST;
    fbsde_problem Pd = *P;
    Layout L;
    int st = make_layout(&Pd, Q, L);
    if (st != FBSDE_OK) return st;
    const size_t Qs = (size_t)Q, ds = (size_t)P->d;
    const size_t need = L.total + fbsde_host_staging_bytes(&Pd, Q);
    if (!workspace || workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) % kAlign))
        return FBSDE_ERR_WORKSPACE;
    if (needs_theta && !P->theta) return FBSDE_ERR_ARG;
    char *stage = static_cast<char *>(workspace) + L.total;
    double *x0_d = reinterpret_cast<double *>(stage);
    double *grad_d = reinterpret_cast<double *>(stage + align_up(Qs * ds * 8, kAlign));
    double *u0_d = reinterpret_cast<double *>(stage + 2 * align_up(Qs * ds * 8, kAlign));
    double *th_d = reinterpret_cast<double *>(stage + 2 * align_up(Qs * ds * 8, kAlign) +
                                              align_up(Qs * 8, kAlign));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(x0_d, x0_host, Qs * ds * 8, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return FBSDE_ERR_CUDA;
    if (needs_theta &&
        cudaMemcpyAsync(th_d, P->theta, ds * 8, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return FBSDE_ERR_CUDA;
    Pd.theta = needs_theta ? th_d : nullptr;
    st = solve_impl(&Pd, Q, x0_d, Pd.theta, seed, solve_index0, u0_d,
                    grad_u0_host ? grad_d : nullptr, nullptr, workspace, L.total, s);
    if (st != FBSDE_OK) return st;
    if (cudaMemcpyAsync(u0_host, u0_d, Qs * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return FBSDE_ERR_CUDA;
    if (grad_u0_host &&
        cudaMemcpyAsync(grad_u0_host, grad_d, Qs * ds * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return FBSDE_ERR_CUDA;
    fbsde_diag dg;
    st = fbsde_diagnostics(&Pd, Q, workspace, &dg, stream);
    return st != FBSDE_OK ? st : dg.status;
}

int fbsde_diagnostics(const fbsde_problem *P, int32_t Q, const void *workspace, fbsde_diag *out,
                      fbsde_stream_t stream)
{
    if (!out) return FBSDE_ERR_ARG;
    Layout L;
    const int st = make_layout(P, Q, L);
    if (st != FBSDE_OK) return st;
    if (!workspace) return FBSDE_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(s) != cudaSuccess) return FBSDE_ERR_CUDA;
    SolveState *h = new (std::nothrow) SolveState[Q];
    if (!h) return FBSDE_ERR_ARG;
    const cudaError_t e = cudaMemcpy(h, static_cast<const char *>(workspace) + L.off_state,
                                     sizeof(SolveState) * Q, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        delete[] h;
        return FBSDE_ERR_CUDA;
    }
    fbsde_diag d{};
    for (int q = 0; q < Q; ++q) {
        if (d.status == FBSDE_OK && h[q].status != 0) d.status = h[q].status;
        d.solves_cg_exhausted += h[q].cg_exhausted ? 1 : 0;
        d.max_newton_iters = std::max(d.max_newton_iters, h[q].newton_max_all);
        d.cg_iters_total += h[q].cg_total;
    }
    delete[] h;
    *out = d;
    return FBSDE_OK;
}

size_t fbsde_plan_workspace_bytes(int32_t n, const fbsde_instance *inst)
{
    std::vector<PlanInstance> v;
    size_t total = 0;
    return plan_layout(n, inst, v, total) == FBSDE_OK ? total : 0;
}

// Scheduling model of a CG pass for the plan's branches: the launches of a pass (product,
// reduction, update) cost about 25 us however small the instance, and its rows stream at
// about 6.5 TB/s.
constexpr double kPassLatency = 25e-6;
constexpr double kPassBandwidth = 6.5e12;

int fbsde_plan_create(fbsde_plan **plan, int32_t n, const fbsde_instance *inst, int32_t branches,
                      void *workspace, size_t workspace_bytes)
{
    if (!plan) return FBSDE_ERR_ARG;
    *plan = nullptr;
    std::vector<PlanInstance> v;
    size_t total = 0;
    int st = plan_layout(n, inst, v, total);
    if (st != FBSDE_OK) return st;
    if (!workspace || workspace_bytes < total || (reinterpret_cast<uintptr_t>(workspace) % kAlign))
        return FBSDE_ERR_WORKSPACE;
    const int B = std::max(1, std::min<int>(n, branches > 0 ? branches : 32));
    fbsde_plan *pl = new (std::nothrow) fbsde_plan();
    if (!pl) return FBSDE_ERR_ARG;
    pl->inst = v;
    pl->workspace = workspace;
    auto fail = [&](cudaError_t) {
        plan_free(pl);
        return (int)FBSDE_ERR_CUDA;
    };
    // streams: 0 = capture origin, 1 = conditional bodies, 2.. = branches
    for (int i = 0; i < B + 2; ++i) {
        cudaStream_t sx;
        if (cudaStreamCreateWithFlags(&sx, cudaStreamNonBlocking) != cudaSuccess) return fail(cudaErrorUnknown);
        pl->streams.push_back(sx);
    }
    for (int i = 0; i < B + 1; ++i) {
        cudaEvent_t ev;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return fail(cudaErrorUnknown);
        pl->events.push_back(ev);
    }
    // largest-first list scheduling of the instances over the branches
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    // time estimate: N levels times the passes per level, 2 + the CG iterations, which
    // grow like the square root of the condition number of the regression (for a cloud
    // of M points in d dimensions, ratio rho = min(d/M, M/d), the extreme eigenvalues
    // are near (1 -+ sqrt(rho))^2, and the ridge bounds the smallest from below), times
    // the time of a pass: a fixed latency of its launches plus its rows at the HBM
    // bandwidth.  Without the latency term the many small instances look free and pile
    // up on a few branches as long chains of latency-bound passes.
    auto cost = [&](int i) {
        const fbsde_problem &P = v[i].in.problem;
        const double rho = std::min((double)P.d / P.M, (double)P.M / P.d);
        const double hi = (1.0 + std::sqrt(rho)) * (1.0 + std::sqrt(rho));
        const double lo = std::max((1.0 - std::sqrt(rho)) * (1.0 - std::sqrt(rho)),
                                   std::max(P.ridge_rel, 1e-6) * hi);
        const double bytes = (double)v[i].in.Q * P.M * P.d * (P.precision == FBSDE_FP32 ? 4 : 8);
        return (double)P.N * (2.0 + std::sqrt(hi / lo)) * (kPassLatency + bytes / kPassBandwidth);
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
    std::vector<double> load(B, 0.0);
    std::vector<std::vector<int>> lists(B);
    for (int i : order) {
        const int b = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        lists[b].push_back(i);
        load[b] += cost(i);
    }
    cudaStream_t origin = pl->streams[0], body = pl->streams[1];
    if (cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return fail(cudaErrorUnknown);
    cudaError_t e = cudaEventRecord(pl->events[0], origin);
    for (int b = 0; b < B && e == cudaSuccess; ++b)
        e = cudaStreamWaitEvent(pl->streams[2 + b], pl->events[0], 0);
    for (int b = 0; b < B && e == cudaSuccess; ++b) {
        const Rec r{pl->streams[2 + b], true, body, false};
        for (int i : lists[b]) {
            const PlanInstance &pi = v[i];
            void *ws = static_cast<char *>(workspace) + pi.offset;
            const Params p = make_params(&pi.in.problem, pi.L, ws, pi.in.seed, pi.in.solve_index0,
                                         pi.in.u0, pi.in.grad_u0, nullptr);
            e = pi.in.problem.precision == FBSDE_FP32
                    ? run<float>(p, pi.L, pi.in.x0, pi.in.problem.theta, r)
                    : run<double>(p, pi.L, pi.in.x0, pi.in.problem.theta, r);
            if (e != cudaSuccess) break;
        }
        if (e == cudaSuccess) e = cudaEventRecord(pl->events[1 + b], pl->streams[2 + b]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(origin, pl->events[1 + b], 0);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(origin, &g);
    pl->graph = g;
    if (e != cudaSuccess || ec != cudaSuccess || !g) return fail(e);
    if (cudaGraphInstantiate(&pl->exec, g, 0) != cudaSuccess) return fail(cudaErrorUnknown);
    *plan = pl;
    return FBSDE_OK;
}

int fbsde_plan_launch(fbsde_plan *plan, fbsde_stream_t stream)
{
    if (!plan || !plan->exec) return FBSDE_ERR_ARG;
    return cudaGraphLaunch(plan->exec, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
               ? FBSDE_OK
               : FBSDE_ERR_CUDA;
}

int fbsde_plan_diagnostics(fbsde_plan *plan, fbsde_diag *out, fbsde_stream_t stream)
{
    if (!plan || !out) return FBSDE_ERR_ARG;
    fbsde_diag acc{};
    for (const PlanInstance &pi : plan->inst) {
        fbsde_diag d{};
        const int st = fbsde_diagnostics(&pi.in.problem, pi.in.Q,
                                         static_cast<char *>(plan->workspace) + pi.offset, &d, stream);
        if (st != FBSDE_OK) return st;
        if (acc.status == FBSDE_OK) acc.status = d.status;
        acc.solves_cg_exhausted += d.solves_cg_exhausted;
        acc.max_newton_iters = std::max(acc.max_newton_iters, d.max_newton_iters);
        acc.cg_iters_total += d.cg_iters_total;
    }
    *out = acc;
    return FBSDE_OK;
}

int fbsde_plan_instance_diagnostics(fbsde_plan *plan, int32_t index, fbsde_diag *out,
                                    fbsde_stream_t stream)
{
    if (!plan || !out || index < 0 || index >= (int32_t)plan->inst.size()) return FBSDE_ERR_ARG;
    const PlanInstance &pi = plan->inst[index];
    return fbsde_diagnostics(&pi.in.problem, pi.in.Q,
                             static_cast<char *>(plan->workspace) + pi.offset, out, stream);
}

void fbsde_plan_destroy(fbsde_plan *plan) { plan_free(plan); }

int fbsde_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int64_t n,
                        fbsde_stream_t stream)
{
    if (!ctr || !key || !out || n < 0) return FBSDE_ERR_ARG;
    if (n == 0) return FBSDE_OK;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    k_philox<<<blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(ctr, key, out, n);
    return cudaGetLastError() == cudaSuccess ? FBSDE_OK : FBSDE_ERR_CUDA;
}

int fbsde_normals(uint64_t seed, uint32_t s, uint32_t k, uint32_t j0, int32_t nj, int32_t d,
                  int32_t precision, void *out, fbsde_stream_t stream)
{
    if (!out || nj < 0 || d < 1) return FBSDE_ERR_ARG;
    if (nj == 0) return FBSDE_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (precision == FBSDE_FP32) e = Launch<float>::normals(seed, s, k, j0, nj, d, out, st);
    else if (precision == FBSDE_FP64) e = Launch<double>::normals(seed, s, k, j0, nj, d, out, st);
    else return FBSDE_ERR_ARG;
    return e == cudaSuccess ? FBSDE_OK : FBSDE_ERR_CUDA;
}

int fbsde_profile_start(int32_t max_timed_launches)
{
    if (max_timed_launches < 0 || max_timed_launches > (1 << 22)) return FBSDE_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    for (cudaEvent_t e : g_prof.ev) cudaEventDestroy(e);
    g_prof.ev.assign(2 * (size_t)max_timed_launches, nullptr);
    g_prof.fam.assign((size_t)max_timed_launches, 0);
    for (auto &e : g_prof.ev)
        if (cudaEventCreate(&e) != cudaSuccess) return FBSDE_ERR_CUDA;
    g_prof.cap = max_timed_launches;
    g_prof.used = 0;
    std::fill(g_prof.launches, g_prof.launches + FBSDE_NUM_KERNELS, 0);
    g_prof.on = true;
    return FBSDE_OK;
}

int fbsde_profile_select(uint32_t family_mask)
{
    const uint32_t all = (1u << FBSDE_NUM_KERNELS) - 1;
    if (!(family_mask & all)) return FBSDE_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    g_prof.mask = family_mask & all;
    return FBSDE_OK;
}

int fbsde_profile_stop(fbsde_kernel_stats *out)
{
    std::lock_guard<std::mutex> lk(g_prof.mu);
    g_prof.on = false;
    g_prof.mask = (1u << FBSDE_NUM_KERNELS) - 1;
    int st = FBSDE_OK;
    fbsde_kernel_stats acc[FBSDE_NUM_KERNELS] = {};
    for (int f = 0; f < FBSDE_NUM_KERNELS; ++f) acc[f].launches = g_prof.launches[f];
    for (int i = 0; i < g_prof.used; ++i) {
        float ms = 0.0f;
        if (cudaEventSynchronize(g_prof.ev[2 * i + 1]) != cudaSuccess ||
            cudaEventElapsedTime(&ms, g_prof.ev[2 * i], g_prof.ev[2 * i + 1]) != cudaSuccess) {
            st = FBSDE_ERR_CUDA;
            continue;
        }
        acc[g_prof.fam[i]].timed += 1;
        acc[g_prof.fam[i]].total_ms += ms;
    }
    for (cudaEvent_t e : g_prof.ev) cudaEventDestroy(e);
    g_prof.ev.clear();
    g_prof.fam.clear();
    g_prof.cap = g_prof.used = 0;
    if (out) std::memcpy(out, acc, sizeof(acc));
    return st;
}

const char *fbsde_kernel_name(int family)
{
    static const char *names[FBSDE_NUM_KERNELS] = {
        "setup", "forward", "update", "matvec", "moments", "reduce",
        "cg_step", "cg_post", "trace", "particles", "finalize", "adjoint", "step"};
    return (family >= 0 && family < FBSDE_NUM_KERNELS) ? names[family] : "unknown";
}

const char *fbsde_status_string(int status)
{
    switch (status) {
    case FBSDE_OK: return "ok";
    case FBSDE_ERR_ARG: return "invalid argument";
    case FBSDE_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case FBSDE_ERR_CUDA: return "CUDA error";
    case FBSDE_ERR_NEWTON: return "Newton iteration did not converge";
    case FBSDE_ERR_CG: return "CG did not reach its tolerance";
    case FBSDE_ERR_TIMEOUT: return "device wait timed out";
    case FBSDE_ERR_NONFINITE: return "non-finite result";
    }
    return "unknown status";
}

int fbsde_check_bounded_wait(int64_t limit_ns, void *scratch, int64_t *waited_ns,
                             fbsde_stream_t stream)
{
    if (limit_ns <= 0 || limit_ns > 1000000000LL || !scratch ||
        (reinterpret_cast<uintptr_t>(scratch) % 8))
        return FBSDE_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned long long h[2] = {0, 0};
    int *out = static_cast<int *>(scratch);
    unsigned long long *ns = reinterpret_cast<unsigned long long *>(static_cast<char *>(scratch) + 8);
    k_wait_probe<<<1, 32, 0, s>>>((unsigned long long)limit_ns, out, ns);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(h, scratch, 16, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return FBSDE_ERR_CUDA;
    if (waited_ns) *waited_ns = (int64_t)h[1];
    return (int)(h[0] & 0xffffffffu);
}

int fbsde_abi_version(void) { return FBSDE_ABI_VERSION; }

}  // extern "C"
