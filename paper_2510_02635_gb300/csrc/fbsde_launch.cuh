// fbsde_launch.cuh -- host launchers of the kernels for one stream precision.
#pragma once
#include "fbsde_kernels.cuh"

namespace fbsde {

// Dynamic shared memory of a streaming kernel: team slots, the CTA reduction buffer
// (multi-team CTAs only) and per-team scalars.
template <typename Real> inline size_t stream_smem(const Layout &L)
{
    size_t b = (size_t)L.teams * 2 * 32 * 4 * sizeof(Real);
    if (L.teams > 1) b += (size_t)L.teams * L.ld * sizeof(Real);
    b += (size_t)L.teams * 3 * sizeof(double) + 16;
    return b;
}

template <typename Real, int VPT, typename K>
static cudaError_t launch_stream(K kernel, const Params &p, const Layout &L, cudaStream_t s)
{
    const size_t smem = stream_smem<Real>(L);
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    kernel<<<dim3(L.G, L.Q), L.threads, smem, s>>>(p, L.Q);
    return cudaGetLastError();
}

#define FBSDE_VPT_DISPATCH(KERNEL)                                                        \
    switch (L.vpt) {                                                                      \
    case 1: return launch_stream<Real, 1>(dev::KERNEL<Real, 1>, p, L, s);                 \
    case 2: return launch_stream<Real, 2>(dev::KERNEL<Real, 2>, p, L, s);                 \
    case 4: return launch_stream<Real, 4>(dev::KERNEL<Real, 4>, p, L, s);                 \
    case 8: return launch_stream<Real, 8>(dev::KERNEL<Real, 8>, p, L, s);                 \
    }                                                                                     \
    return cudaErrorInvalidValue;

template <typename Real>
cudaError_t Launch<Real>::setup(const Params &p, const double *x0, const double *theta, int Q,
                                cudaStream_t s)
{
    dev::k_setup<Real><<<Q, kFinThreads, 0, s>>>(p, x0, theta, Q);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t Launch<Real>::forward(const Params &p, const Layout &L, cudaStream_t s)
{
    FBSDE_VPT_DISPATCH(k_forward)
}

template <typename Real>
cudaError_t Launch<Real>::update(const Params &p, const Layout &L, cudaStream_t s)
{
    FBSDE_VPT_DISPATCH(k_update)
}

template <typename Real>
cudaError_t Launch<Real>::matvec(const Params &p, const Layout &L, cudaStream_t s)
{
    FBSDE_VPT_DISPATCH(k_matvec)
}

template <typename Real>
cudaError_t Launch<Real>::moments_finalize(const Params &p, const Layout &L, cudaStream_t s)
{
    dev::k_moments_finalize<Real><<<L.Q, kFinThreads, 0, s>>>(p, p.has_r);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t Launch<Real>::cg_start(const Params &p, const Layout &L, cudaStream_t s)
{
    dev::k_cg_start<Real><<<L.Q, kFinThreads, 0, s>>>(p);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t Launch<Real>::cg_finalize(const Params &p, const Layout &L, cudaStream_t s)
{
    dev::k_cg_finalize<Real><<<L.Q, kFinThreads, 0, s>>>(p);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t Launch<Real>::cg_post(const Params &p, const Layout &L, cudaStream_t s)
{
    dev::k_cg_post<Real><<<L.Q, kFinThreads, 0, s>>>(p);
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

}  // namespace fbsde
