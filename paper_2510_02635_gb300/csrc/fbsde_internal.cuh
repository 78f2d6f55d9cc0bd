// fbsde_internal.cuh -- shared declarations of the CUDA implementation (not part of the ABI).
//
// Data layout in HBM (one workspace, caller-allocated, 256-byte aligned sections):
//   delta  [Q][M][ld]      Real   particle displacement X_k^j - x0 of the current level
//   Y      [Q][M]          double Y_k^j of the current level
//   w      [Q][M]          Real   kernel weight of particle j in the current regression
//   coef   [Q][M][3]       Real   moment coefficients (w, w (Y - yref), w D.x_ws)
//   segp   [Q][M][nseg][6] Real   per-row-segment partial sums of the row kernels
//   part   [Q][G][3][ld]   Real   per-CTA partial d-vectors (moments or the CG product)
//   spart  [Q][GS][4]      double per-particle-block partial scalars
//   vec64  [Q][9][ld]      double x (= alpha_x), r, p, S, b/rhs, q/G, x0, s, previous alpha_x
//   vecR   [Q][4][ld]      Real   p, alpha_x, x0, next starting guess (stream precision);
//                                 then theta [ld]
//   state  [Q]             SolveState
// and, for a forward SDE with a drift or a state-dependent diffusion only:
//   store  [slots][Q][M][ld] Real stored levels of the rows (checkpoints, one segment)
//   anchor [Q][N+1][ld]    Real   offsets c_k = a_k - x0 of the drift path of x0
// ld = d rounded up to a multiple of 4 (16-byte rows for float and 32-byte rows for
// double); the padding of every row and vector is kept at zero.
#pragma once
#include <cmath>
#include <cstddef>
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/fbsde.h"

namespace fbsde {

// fbsde_solve with every CG pass launched on the stream, creating no CUDA graph
// (fbsde_api.cu); used by the entry point without a workspace argument.
int solve_launches_only(const fbsde_problem *P, int32_t Q, const double *x0, uint64_t seed,
                        uint32_t solve_index0, double *u0, double *grad_u0, void *workspace,
                        size_t workspace_bytes, cudaStream_t stream);

constexpr int kPartVecs = 3;
constexpr int kPartScal = 4;
constexpr int kVec64 = 9;
constexpr int kRedTile = 128;  // elements per block of the partial reduction and CG update
constexpr int kBpart = 4;      // per-block shares: w . r, S . r, r . r, spare
constexpr int kVecR = 4;
constexpr int kSegSums = 6;   // per-row-segment sums of the row kernels (the forward SDE's
                              // rows use all six, the driftless ones the first four)
constexpr int kFinThreads = 512;   // threads of the one-CTA-per-solve kernels
constexpr int kTargetCtas = 608;   // default: 4 x 152 SMs, CTAs of one streaming pass over all queries
constexpr int kMinRowsPerCta = 32;   // rows of a streaming pass per CTA at least: fewer
                                     // partial vectors for the reduction of small clouds
constexpr int kRowBlocks = 152 * 8;  // grid of the row-segment kernels (grid-stride)
constexpr int kStepMaxLd = 10240;    // widest FP32 row of the fused per-level step
constexpr int kStepElems = 10240;    // particle-dims per stage of the fused step

struct SolveState {
    double c, alpha, lambda, invW, rr, rhs2, sp, yref, sumz, zz, phi0, gx0;
    double abar, sv, sumz_l, zz_l;  // reverse sweep
    double rr_prev, cg_alpha;       // previous r . r and step of the CG recurrence
    double sx;                      // S . x of the adjoint solve's starting guess
    double rho_ref;                 // forward SDE: mean squared distance to the anchor
    double sum_ax, ax_x0;           // forward SDE: sum_i alpha_x,i and alpha_x . x0
    double psi0;                    // forward SDE: second feature of f at x0 (kinds 7, 8)
    int32_t iters, done, status, newton_max, cg_exhausted, newton_max_all, loop_iter, cg_total, arrive,
        arrive_q;
};

struct Layout {
    int Q, d, ld, N, G, precision, team_warps, vpt, teams, threads;
    size_t off_tape_w, off_tape_Y, off_tape_v, off_tape_s, off_adj_v, total_adjoint;
    int seg_vpt, nseg, GP, mom_vm, mom_tiles, row_blocks, mv_rows, mv_stages, red_groups, nblk;
    size_t mv_smem;
    // fused per-level step (FP32 rows of at most kStepMaxLd floats): rows per stage, threads
    // per row, chunks per thread in the row pass, column-pass row groups, shared memory
    int fused, st_R, st_T, st_vm1, st_tpr, st_RG, st_vm3, st_vm, st_nslot, GS, Gs;
    // forward SDE with drift / state-dependent diffusion: checkpoint interval s, checkpoint
    // slabs, slabs in all (checkpoints, then one segment), stored rows and anchor offsets
    int sde, sde_s, sde_ncp, sde_slots;
    size_t off_store, off_anchor;
    size_t st_region, st_smem;
    int64_t M;
    size_t real_sz;
    size_t off_delta, off_Y, off_w, off_coef, off_segp, off_part, off_spart, off_vec64, off_vecR,
        off_state, off_bpart;
    size_t total;
};

// Everything a kernel needs, passed by value.
struct Params {
    // problem
    int kind, d, ld, N, G, team_warps, level, uniform, cg_max_iter, newton_max_iter, has_r,
        newton_level, Q, nseg, GP, GS, mv_rows, mv_stages, walk, nblk;
    long long M;
    double sigma, T, dt, sdt, A, c0, c1, c2, c3, h2, ridge_rel, cg_tol2, newton_tol;
    double wa, wb;  // path step of the row kernels: Delta <- wa Delta + wb xi (set per launch)
    int st_R, st_T, st_vm1, st_tpr, st_RG, st_vm3, st_nslot, nsp;  // fused step geometry;
                                                                    // nsp = spart blocks of a level
    long long st_region;  // floats of the fused step's row-slot region
    uint32_t rk0[10], rk1[10];  // Philox4x32-10 round keys of (key0, key1)
    // forward SDE: mu_i(x) = mu0 + mu1 x_i, sigma_ii(x) = sigma + sig1 x_i; anchor offsets
    // c_k = a_k - x0 [Q][N+1][ld] (stream precision)
    int sde;
    double mu0, mu1, sig1;
    void *anchor;
    uint32_t key0, key1, solve0;
    // workspace
    void *delta;
    double *Y;
    void *w;
    void *coef;
    void *segp;
    void *part;
    double *spart;
    double *vec64;
    void *vecR;
    SolveState *st;
    double *bpart;  // [Q][nblk][kBpart] per-block shares of the CG dot products
    // tape of the primal for the reverse sweep (null when not recording)
    void *tape_w;
    double *tape_Y, *tape_v, *tape_s, *adj_v;
    const double *theta;
    // outputs
    double *u0, *grad;
    double *tr_alpha, *tr_alpha_x, *tr_x_N, *tr_y_N;
    int32_t *tr_cg, *tr_newton;
};

// Host-side launchers, one set per stream precision (fbsde_launch.cuh).
template <typename Real> struct Launch {
    static cudaError_t setup(const Params &p, const double *x0, const double *theta, cudaStream_t s);
    static cudaError_t forward(const Params &p, const Layout &L, cudaStream_t s);
    static cudaError_t update(const Params &p, const Layout &L, cudaStream_t s);
    static cudaError_t particles(const Params &p, const Layout &L, cudaStream_t s);
    static cudaError_t moments(const Params &p, const Layout &L, cudaStream_t s);
    static cudaError_t step(const Params &p, const Layout &L, cudaStream_t s);
    // forward SDE (fbsde_sde.cuh)
    static cudaError_t sde_anchor(const Params &p, const Layout &L, cudaStream_t s);
    static cudaError_t sde_forward(const Params &p, const Layout &L, int k, const void *from,
                                   void *to, cudaStream_t s);
    static cudaError_t sde_rows(const Params &p, const Layout &L, int k, const void *src,
                                cudaStream_t s);
    static cudaError_t sde_rho(const Params &p, const Layout &L, cudaStream_t s);
    static cudaError_t reduce(const Params &p, const Layout &L, int nvec, int dst0, int skip_done,
                              cudaStream_t s);
    static cudaError_t matvec(const Params &p, const Layout &L, cudaStream_t s);
    static cudaError_t moments_finalize(const Params &p, const Layout &L, int warm, cudaStream_t s);
    static cudaError_t cg_update(const Params &p, const Layout &L, cudaGraphConditionalHandle h,
                               int use_h, cudaStream_t s);
    static cudaError_t cg_post(const Params &p, const Layout &L, cudaStream_t s);
    static cudaError_t cg_reset(const Params &p, cudaGraphConditionalHandle h, cudaStream_t s);
    static cudaError_t trace_forward(const Params &p, const Layout &L, cudaStream_t s);
    static cudaError_t normals(uint64_t seed, uint32_t s, uint32_t k, uint32_t j0, int nj, int d,
                               void *out, cudaStream_t st);
    // reverse sweep
    static cudaError_t adj_init(const Params &p, const Layout &L, const double *ubar, cudaStream_t s);
    static cudaError_t adj_warm(const Params &p, const Layout &L, cudaStream_t s);
    static cudaError_t adj_setup(const Params &p, const Layout &L, int warm, cudaStream_t s);
    static cudaError_t adj_post(const Params &p, const Layout &L, cudaStream_t s);
    static cudaError_t adj_rows(const Params &p, const Layout &L, cudaStream_t s);
    static cudaError_t adj_zlevel(const Params &p, const Layout &L, cudaStream_t s);
    static cudaError_t adj_particles(const Params &p, const Layout &L, cudaStream_t s);
    static cudaError_t adj_colsum(const Params &p, const Layout &L, int mode_b, int mode_c,
                                  cudaStream_t s);
    static cudaError_t adj_finalize(const Params &p, const Layout &L, cudaStream_t s);
    static cudaError_t adj_output(const Params &p, const Layout &L, double *x0bar, double *thetabar,
                                  cudaStream_t s);
};



}  // namespace fbsde
