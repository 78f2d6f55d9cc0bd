// Check of the tensor-core products k_gemm_tc (split TF32, tcgen05) against FP64 host
// products of the same FP32 inputs, on ragged shapes of both layouts (k contiguous, "NT",
// and rows contiguous, "TN", split over K).  Prints one line per shape and exits 1 when an
// element's error exceeds 4e-6 of sum_k |a b|, or a kernel reports a status.
#include <algorithm>
#include <cmath>
#include <cstdio>
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

int main()
{
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
