// Check of the tensor-core products k_gemm_tc (split TF32, tcgen05) against FP64 host
// products of the same FP32 inputs, on ragged shapes of both layouts (k contiguous, "NT",
// and rows contiguous, "TN", split over K).  Prints one line per shape and exits 1 when an
// element's error exceeds 4e-6 of sum_k |a b|, or a kernel reports a status.
// With arguments "time M d": times, with CUDA events over 20 launches after 3 warm-up
// launches, the two products of a per-anchor CG pass at M particles in d dimensions (row
// stride ld = d rounded up to 4): P V^T (NT, M x M x ld) and T^T P (TN, M x ld x M, split
// over the particles by the solve's rule), plain launches for a profiler.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "fbsde_tcgemm.cuh"

using fbsde::dev::k_gemm_tc;
using fbsde::dev::kTcSmemBytes;
using fbsde::dev::kTcThreads;
using fbsde::dev::TcStore;

namespace {

uint64_t rs = 88172645463325252ull;   // xorshift64 inputs
double urand()
{
    rs ^= rs << 13;
    rs ^= rs >> 7;
    rs ^= rs << 17;
    return (double)(rs >> 11) * 0x1p-53;
}

struct Case {
    bool tn;
    int Mr, Nc, K, kc;
};

template <bool TN>
cudaError_t launch(const Case &c, const float *A, int lda, const float *B, int ldb, float *C,
                   int ldc, int *st)
{
    cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<TN, TcStore>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTcSmemBytes);
    if (e != cudaSuccess) return e;
    const dim3 grid((c.Nc + 127) / 128, (c.Mr + 127) / 128, (c.K + c.kc - 1) / c.kc);
    k_gemm_tc<TN, TcStore><<<grid, kTcThreads, kTcSmemBytes>>>(c.Mr, c.Nc, c.K, c.kc, A, lda, B,
                                                              ldb, TcStore{C, c.Mr, ldc}, st, fbsde::dev::Band{0, 0});
    return cudaGetLastError();
}

}  // namespace

// K splits of the solve's tall products (about two waves of 64 x 64 tiles, at least 128
// rows per split, split lengths multiples of 16).
int solve_kc(int M, int ld)
{
    const long long tiles = ((long long)(ld + 63) / 64) * ((M + 63) / 64);
    const long long want = std::max(1ll, (2ll * 152 * 4 + tiles - 1) / tiles);
    const long long ns = std::max(1ll, std::min(want, (long long)(M / 128)));
    return (int)(((M + ns - 1) / ns + 15) / 16 * 16);
}

int time_products(int M, int d)
{
    const int ld = (d + 3) / 4 * 4, kc = solve_kc(M, ld), ns = (M + kc - 1) / kc;
    const size_t np = (size_t)M * ld, nt = (size_t)M * M, ng = (size_t)ns * M * ld;
    std::vector<float> h(std::max(np, nt));
    float *P = nullptr, *V = nullptr, *T = nullptr, *U = nullptr, *G = nullptr;
    int *st = nullptr;
    if (cudaMalloc(&P, np * 4) || cudaMalloc(&V, np * 4) || cudaMalloc(&T, nt * 4) ||
        cudaMalloc(&U, nt * 4) || cudaMalloc(&G, ng * 4) || cudaMalloc(&st, sizeof(int)))
        return 2;
    for (size_t i = 0; i < np; ++i) h[i] = (float)(2 * urand() - 1);
    cudaMemcpy(P, h.data(), np * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(V, h.data(), np * 4, cudaMemcpyHostToDevice);
    for (size_t i = 0; i < nt; ++i) h[i] = (float)urand() * 1e-3f;
    cudaMemcpy(T, h.data(), nt * 4, cudaMemcpyHostToDevice);
    cudaMemset(st, 0, sizeof(int));
    const Case nt_case{false, M, M, ld, ld}, tn_case{true, M, ld, M, kc};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int which = 0; which < 2; ++which) {
        const Case &c = which ? tn_case : nt_case;
        float ms = 0.0f;
        cudaError_t e = cudaSuccess;
        for (int it = 0; it < 23 && e == cudaSuccess; ++it) {
            if (it == 3) cudaEventRecord(e0);
            e = which ? launch<true>(c, T, M, P, ld, G, ld, st)
                      : launch<false>(c, P, ld, V, ld, U, M, st);
        }
        cudaEventRecord(e1);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            printf("CUDA error %s\n", cudaGetErrorString(e));
            return 2;
        }
        cudaEventElapsedTime(&ms, e0, e1);
        const double us = 1e3 * ms / 20, flop = 2.0 * M * (double)M * ld;
        printf("%s M=%d ld=%d splits=%d: %.1f us per launch, %.1f TF/s useful, %.1f TF/s "
               "executed (3 TF32 MMAs per useful one)\n",
               which ? "TN T^T P" : "NT P V^T", M, ld, which ? ns : 1, us, flop / us * 1e-6,
               3 * flop / us * 1e-6);
    }
    int hst = 0;
    cudaMemcpy(&hst, st, sizeof(int), cudaMemcpyDeviceToHost);
    printf("status %d\n", hst);
    cudaFree(P);
    cudaFree(V);
    cudaFree(T);
    cudaFree(U);
    cudaFree(G);
    cudaFree(st);
    return hst ? 1 : 0;
}

int main(int argc, char **argv)
{
    if (argc == 4 && std::string(argv[1]) == "time") {
        const int M = std::atoi(argv[2]), d = std::atoi(argv[3]);
        if (M < 128 || M > 32768 || d < 1 || d > 16384) return 2;
        return time_products(M, d);
    }
    const Case cases[] = {{false, 150, 150, 100, 100},  {false, 1030, 1030, 24, 24},
                          {false, 2048, 300, 104, 104}, {false, 200, 130, 4, 4},
                          {true, 2048, 104, 2048, 128}, {true, 1030, 24, 1030, 144},
                          {true, 300, 70, 250, 100}};
    int *st = nullptr;
    if (cudaMalloc(&st, sizeof(int)) != cudaSuccess) return 2;
    cudaMemset(st, 0, sizeof(int));
    int bad = 0;
    for (const Case &c : cases) {
        const int ns = (c.K + c.kc - 1) / c.kc;
        const size_t na = (size_t)c.K * c.Mr, nb = (size_t)c.K * c.Nc, nc = (size_t)ns * c.Mr * c.Nc;
        std::vector<float> a(na), b(nb), out(nc);
        for (float &x : a) x = (float)((2 * urand() - 1) * std::ldexp(1.0, (int)(urand() * 8) - 4));
        for (float &x : b) x = (float)(2 * urand() - 1);
        float *dA = nullptr, *dB = nullptr, *dC = nullptr;
        if (cudaMalloc(&dA, na * 4) || cudaMalloc(&dB, nb * 4) || cudaMalloc(&dC, nc * 4)) return 2;
        cudaMemcpy(dA, a.data(), na * 4, cudaMemcpyHostToDevice);
        cudaMemcpy(dB, b.data(), nb * 4, cudaMemcpyHostToDevice);
        cudaMemset(dC, 0xFF, nc * 4);   // NaN: every element must be written
        const int lda = c.tn ? c.Mr : c.K, ldb = c.tn ? c.Nc : c.K, ldc = c.Nc;
        cudaError_t e = c.tn ? launch<true>(c, dA, lda, dB, ldb, dC, ldc, st)
                             : launch<false>(c, dA, lda, dB, ldb, dC, ldc, st);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
            printf("CUDA error %s\n", cudaGetErrorString(e));
            return 2;
        }
        cudaMemcpy(out.data(), dC, nc * 4, cudaMemcpyDeviceToHost);
        double worst = 0.0;
        for (int z = 0; z < ns; ++z) {
            const int k0 = z * c.kc, k1 = std::min(c.K, k0 + c.kc);
            for (int r = 0; r < c.Mr; ++r)
                for (int n = 0; n < c.Nc; ++n) {
                    double s = 0.0, sa = 0.0;
                    for (int k = k0; k < k1; ++k) {
                        const double x = c.tn ? a[(size_t)k * lda + r] : a[(size_t)r * lda + k];
                        const double y = c.tn ? b[(size_t)k * ldb + n] : b[(size_t)n * ldb + k];
                        s += x * y;
                        sa += std::fabs(x * y);
                    }
                    const double err =
                        std::fabs((double)out[((size_t)z * c.Mr + r) * ldc + n] - s) / (sa + 1e-30);
                    worst = std::isnan(err) ? INFINITY : std::max(worst, err);
                }
        }
        const bool ok = worst < 4e-6;
        printf("%s Mr=%d Nc=%d K=%d kc=%d splits=%d max_rel_err=%.3e %s\n", c.tn ? "TN" : "NT",
               c.Mr, c.Nc, c.K, c.kc, ns, worst, ok ? "ok" : "BAD");
        bad |= !ok;
        cudaFree(dA);
        cudaFree(dB);
        cudaFree(dC);
    }
    int hst = 0;
    cudaMemcpy(&hst, st, sizeof(int), cudaMemcpyDeviceToHost);
    printf("status %d\n", hst);
    return (bad || hst) ? 1 : 0;
}
