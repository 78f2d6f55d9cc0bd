// fbsde_launch.cuh -- host launchers of the kernels for one stream precision.
#pragma once
#include "fbsde_adjoint.cuh"
#include "fbsde_kernels.cuh"
#include "fbsde_matvec.cuh"
#include "fbsde_sde.cuh"
#include "fbsde_step.cuh"

namespace fbsde {

template <typename K> static cudaError_t set_smem(K kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename Real>
cudaError_t Launch<Real>::setup(const Params &p, const double *x0, const double *theta,
                                cudaStream_t s)
{
    dev::k_setup<Real><<<p.Q, kFinThreads, 0, s>>>(p, x0, theta);
    return cudaGetLastError();
}

#define FBSDE_SEG_DISPATCH(KERNEL, P)                                                     \
    switch (L.seg_vpt) {                                                                  \
    case 1: dev::KERNEL<Real, 1><<<L.row_blocks, 256, 0, s>>>(P); break;                 \
    case 2: dev::KERNEL<Real, 2><<<L.row_blocks, 256, 0, s>>>(P); break;                 \
    case 4: dev::KERNEL<Real, 4><<<L.row_blocks, 256, 0, s>>>(P); break;                 \
    default: return cudaErrorInvalidValue;                                                \
    }                                                                                     \
    return cudaGetLastError();

// Forward sweep: Delta_N = sigma sqrt(T) xi_N, the end point of the Brownian path.
template <typename Real>
cudaError_t Launch<Real>::forward(const Params &p, const Layout &L, cudaStream_t s)
{
    Params q = p;
    q.wa = 0.0;
    q.wb = p.sigma * std::sqrt(p.T);
    FBSDE_SEG_DISPATCH(k_forward, q)
}

// Brownian-bridge step of level k = p.level (1 <= k < N): with W(0) = 0, W(t_k) given
// W(t_{k+1}) is N((t_k/t_{k+1}) W(t_{k+1}), t_k dt / t_{k+1} I), so on the rows
//   walk = -1: Delta_k = a Delta_{k+1} + b xi_k,  a = k/(k+1), b = sigma sqrt(dt k/(k+1));
//   walk = +1: the same step solved for Delta_{k+1} = (Delta_k - b xi_k) / a.
template <typename Real>
cudaError_t Launch<Real>::update(const Params &p, const Layout &L, cudaStream_t s)
{
    if (p.level < 1 || p.level >= p.N) return cudaErrorInvalidValue;
    Params q = p;
    const double a = (double)p.level / (double)(p.level + 1);
    const double b = p.sigma * std::sqrt(p.dt * a);
    q.wa = p.walk < 0 ? a : 1.0 / a;
    q.wb = p.walk < 0 ? b : -b / a;
    FBSDE_SEG_DISPATCH(k_update, q)
}

// Forward SDE with a drift or a state-dependent diffusion (fbsde_sde.cuh).
template <typename Real>
cudaError_t Launch<Real>::sde_anchor(const Params &p, const Layout &L, cudaStream_t s)
{
    const long long n = (long long)L.Q * L.ld;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 1024);
    dev::k_sde_anchor<Real><<<blocks, 256, 0, s>>>(p);
    return cudaGetLastError();
}

// Euler-Maruyama step k -> k + 1 (0 <= k < N) from the rows `from` (nullptr: Delta_0 = 0)
// into `to` (may equal `from`), each [Q][M][ld].
template <typename Real>
cudaError_t Launch<Real>::sde_forward(const Params &p, const Layout &L, int k, const void *from,
                                      void *to, cudaStream_t s)
{
    if (k < 0 || k >= p.N || !to) return cudaErrorInvalidValue;
    const Real *src = static_cast<const Real *>(from);
    Real *dst = static_cast<Real *>(to);
    switch (L.seg_vpt) {
    case 1: dev::k_sde_forward<Real, 1><<<L.row_blocks, 256, 0, s>>>(p, k, src, dst); break;
    case 2: dev::k_sde_forward<Real, 2><<<L.row_blocks, 256, 0, s>>>(p, k, src, dst); break;
    case 4: dev::k_sde_forward<Real, 4><<<L.row_blocks, 256, 0, s>>>(p, k, src, dst); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Row sums of level k from the row buffer, or (src) from a stored level, copied into the
// row buffer on the way.
template <typename Real>
cudaError_t Launch<Real>::sde_rows(const Params &p, const Layout &L, int k, const void *src,
                                   cudaStream_t s)
{
    if (k < 1 || k > p.N) return cudaErrorInvalidValue;
    const Real *sr = static_cast<const Real *>(src);
    switch (L.seg_vpt) {
    case 1: dev::k_sde_rows<Real, 1><<<L.row_blocks, 256, 0, s>>>(p, k, sr); break;
    case 2: dev::k_sde_rows<Real, 2><<<L.row_blocks, 256, 0, s>>>(p, k, sr); break;
    case 4: dev::k_sde_rows<Real, 4><<<L.row_blocks, 256, 0, s>>>(p, k, sr); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename Real>
cudaError_t Launch<Real>::sde_rho(const Params &p, const Layout &L, cudaStream_t s)
{
    dev::k_sde_rho<Real><<<L.Q, kFinThreads, 0, s>>>(p);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t Launch<Real>::particles(const Params &p, const Layout &L, cudaStream_t s)
{
    dev::k_particles<Real><<<dim3(L.GP, L.Q), 256, 0, s>>>(p);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t Launch<Real>::moments(const Params &p, const Layout &L, cudaStream_t s)
{
    const dim3 grid(L.mom_tiles, L.G, L.Q);
    const size_t smem = (size_t)3 * 256 * L.mom_vm * 16;
    cudaError_t e;
    if (L.mom_vm == 1) {
        if ((e = set_smem(dev::k_moments<Real, 1>, smem)) != cudaSuccess) return e;
        dev::k_moments<Real, 1><<<grid, 256, smem, s>>>(p);
    } else {
        if ((e = set_smem(dev::k_moments<Real, 2>, smem)) != cudaSuccess) return e;
        dev::k_moments<Real, 2><<<grid, 256, smem, s>>>(p);
    }
    return cudaGetLastError();
}

// Fused per-level step (FP32 rows of at most kStepMaxLd floats): level k = p.level, with
// 1 <= k < N the Brownian-bridge step Delta_k = a Delta_{k+1} + b xi_k (a = k/(k+1),
// b = sigma sqrt(dt k/(k+1)), as in update), and k = N the end point
// Delta_N = sigma sqrt(T) xi_N of the forward sweep.
template <int VM, bool COSF, bool TERM, bool ONE>
static cudaError_t launch_step(const Params &q, const Layout &L, cudaStream_t s)
{
    cudaError_t e = set_smem(dev::k_step<VM, COSF, TERM, ONE>, L.st_smem);
    if (e != cudaSuccess) return e;
    dev::k_step<VM, COSF, TERM, ONE><<<dim3(q.G, L.Q), dev::kStepThreads, L.st_smem, s>>>(q);
    return cudaGetLastError();
}

template <int VM, bool ONE>
static cudaError_t launch_step_kind(const Params &q, const Layout &L, bool term, bool cosf,
                                    cudaStream_t s)
{
    if (term) return launch_step<VM, false, true, ONE>(q, L, s);
    return cosf ? launch_step<VM, true, false, ONE>(q, L, s)
                : launch_step<VM, false, false, ONE>(q, L, s);
}

template <typename Real>
cudaError_t Launch<Real>::step(const Params &p, const Layout &L, cudaStream_t s)
{
    if constexpr (sizeof(Real) != sizeof(float)) {
        return cudaErrorInvalidValue;
    } else {
        if (!L.fused || p.level < 1 || p.level > p.N) return cudaErrorInvalidValue;
        Params q = p;
        if (p.level == p.N) {
            q.wa = 0.0;
            q.wb = p.sigma * std::sqrt(p.T);
        } else {
            const double a = (double)p.level / (double)(p.level + 1);
            q.wa = a;
            q.wb = p.sigma * std::sqrt(p.dt * a);
        }
        const bool term = p.level == p.N;
        const bool cosf = !term && p.kind == FBSDE_AC_MANUFACTURED;
#define FBSDE_STEP_CASE(VM)                                                              \
    case VM:                                                                             \
        return L.st_R == 1 ? launch_step_kind<VM, true>(q, L, term, cosf, s)             \
                           : launch_step_kind<VM, false>(q, L, term, cosf, s);
        switch (L.st_vm) {
            FBSDE_STEP_CASE(1)
            FBSDE_STEP_CASE(2)
            FBSDE_STEP_CASE(3)
            FBSDE_STEP_CASE(4)
            FBSDE_STEP_CASE(5)
            FBSDE_STEP_CASE(6)
        }
#undef FBSDE_STEP_CASE
        return cudaErrorInvalidValue;
    }
}

template <typename Real>
cudaError_t Launch<Real>::reduce(const Params &p, const Layout &L, int nvec, int dst0,
                                 int skip_done, cudaStream_t s)
{
    dev::k_reduce_partials<Real><<<dim3(L.nblk, L.Q), 32 * L.red_groups, 0, s>>>(p, nvec, dst0,
                                                                                 skip_done);
    return cudaGetLastError();
}

template <typename Real, int VPT, bool WIDE>
static cudaError_t launch_matvec(const Params &p, const Layout &L, cudaStream_t s)
{
    cudaError_t e = set_smem(dev::k_matvec<Real, VPT, WIDE>, L.mv_smem);
    if (e != cudaSuccess) return e;
    dev::k_matvec<Real, VPT, WIDE>
        <<<dim3(L.G, L.Q), 32 * (1 + L.teams * L.team_warps), L.mv_smem, s>>>(p);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t Launch<Real>::matvec(const Params &p, const Layout &L, cudaStream_t s)
{
    const bool wide = 32 * (1 + L.teams * L.team_warps) > 352;
    switch (L.vpt) {
    case 1: return launch_matvec<Real, 1, false>(p, L, s);
    case 2: return launch_matvec<Real, 2, false>(p, L, s);
    case 4: return launch_matvec<Real, 4, false>(p, L, s);
    case 8: return wide ? launch_matvec<Real, 8, true>(p, L, s)
                        : launch_matvec<Real, 8, false>(p, L, s);
    case 16:   // FP64 rows of 8193 to 10240 values: teams of 9 or 10 warps
        if constexpr (sizeof(Real) == 8) {
            if (!wide) return launch_matvec<Real, 16, false>(p, L, s);
        }
        return cudaErrorInvalidValue;
    }
    return cudaErrorInvalidValue;
}

template <typename Real>
cudaError_t Launch<Real>::moments_finalize(const Params &p, const Layout &L, int warm,
                                           cudaStream_t s)
{
    dev::k_moments_finalize<Real><<<L.Q, kFinThreads, 0, s>>>(p, warm);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t Launch<Real>::cg_update(const Params &p, const Layout &L, cudaGraphConditionalHandle h,
                                    int use_h, cudaStream_t s)
{
    dev::k_cg_update<Real><<<dim3(L.nblk, L.Q), 32, 0, s>>>(p, h, use_h);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t Launch<Real>::cg_post(const Params &p, const Layout &L, cudaStream_t s)
{
    dev::k_cg_post<Real><<<L.Q, kFinThreads, 0, s>>>(p);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t Launch<Real>::cg_reset(const Params &p, cudaGraphConditionalHandle h, cudaStream_t s)
{
    dev::k_cg_reset<Real><<<1, 32, 0, s>>>(p, h);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t Launch<Real>::trace_forward(const Params &p, const Layout &L, cudaStream_t s)
{
    const long long n = (long long)p.M * p.d;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
    dev::k_trace_forward<Real><<<dim3(blocks, L.Q), 256, 0, s>>>(p);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t Launch<Real>::normals(uint64_t seed, uint32_t sidx, uint32_t k, uint32_t j0, int nj,
                                  int d, void *out, cudaStream_t st)
{
    dev::k_normals<Real><<<1024, 256, 0, st>>>(seed, sidx, k, j0, nj, d,
                                                reinterpret_cast<Real *>(out));
    return cudaGetLastError();
}

template <typename Real>
cudaError_t Launch<Real>::adj_init(const Params &p, const Layout &L, const double *ubar, cudaStream_t s)
{
    dev::k_adj_init<Real><<<L.Q, kFinThreads, 0, s>>>(p, ubar);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t Launch<Real>::adj_warm(const Params &p, const Layout &L, cudaStream_t s)
{
    dev::k_adj_warm<Real><<<L.Q, kFinThreads, 0, s>>>(p);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t Launch<Real>::adj_setup(const Params &p, const Layout &L, int warm, cudaStream_t s)
{
    dev::k_adj_setup<Real><<<L.Q, kFinThreads, 0, s>>>(p, warm);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t Launch<Real>::adj_post(const Params &p, const Layout &L, cudaStream_t s)
{
    dev::k_adj_post<Real><<<L.Q, kFinThreads, 0, s>>>(p);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t Launch<Real>::adj_rows(const Params &p, const Layout &L, cudaStream_t s)
{
    FBSDE_SEG_DISPATCH(k_adj_rows, p)
}

template <typename Real>
cudaError_t Launch<Real>::adj_zlevel(const Params &p, const Layout &L, cudaStream_t s)
{
    dev::k_adj_zlevel<Real><<<L.Q, kFinThreads, 0, s>>>(p);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t Launch<Real>::adj_particles(const Params &p, const Layout &L, cudaStream_t s)
{
    dev::k_adj_particles<Real><<<dim3(L.GP, L.Q), 256, 0, s>>>(p);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t Launch<Real>::adj_colsum(const Params &p, const Layout &L, int mode_b, int mode_c,
                                     cudaStream_t s)
{
    const dim3 grid(L.mom_tiles, L.G, L.Q);
    const size_t smem = (size_t)3 * 256 * L.mom_vm * 16;
    cudaError_t e;
    if (L.mom_vm == 1) {
        if ((e = set_smem(dev::k_adj_colsum<Real, 1>, smem)) != cudaSuccess) return e;
        dev::k_adj_colsum<Real, 1><<<grid, 256, smem, s>>>(p, mode_b, mode_c);
    } else {
        if ((e = set_smem(dev::k_adj_colsum<Real, 2>, smem)) != cudaSuccess) return e;
        dev::k_adj_colsum<Real, 2><<<grid, 256, smem, s>>>(p, mode_b, mode_c);
    }
    return cudaGetLastError();
}

template <typename Real>
cudaError_t Launch<Real>::adj_finalize(const Params &p, const Layout &L, cudaStream_t s)
{
    dev::k_adj_finalize<Real><<<L.Q, kFinThreads, 0, s>>>(p);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t Launch<Real>::adj_output(const Params &p, const Layout &L, double *x0bar,
                                     double *thetabar, cudaStream_t s)
{
    dev::k_adj_output<Real><<<64, 256, 0, s>>>(p, x0bar, thetabar);
    return cudaGetLastError();
}

}  // namespace fbsde
