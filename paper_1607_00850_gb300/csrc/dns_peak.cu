// Measured FP64 fused-multiply-add throughput of the current device
// (dns_fp64_fma_rate in include/dns.h): the denominator of the FP64 path's
// arithmetic roofline, taken on the GPU the solver runs on instead of a
// nominal data-sheet figure.
//
// Every thread runs kChains independent FMA chains a <- a * b + c (b, c are
// kernel arguments, so nothing folds at compile time), enough independent
// work per warp to cover the FMA latency; the grid holds several blocks per
// SM.  One launch with a short loop calibrates the loop count, a second one
// of about `seconds` is timed with CUDA events.  The chains' sum goes to a
// device variable only if it equals an impossible value, which keeps the
// arithmetic alive without a store per thread.
#include "dns.h"

#include <cuda_runtime.h>

#include <cmath>

namespace {

constexpr int kChains = 16;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;

__device__ double g_peak_sink;

__global__ void __launch_bounds__(kThreads) k_dfma_rate(long long iters, double b, double c) {
    double a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = 1.0 + 1e-3 * threadIdx.x + 1e-6 * i;
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    if (s == -1.0) g_peak_sink = s;  // never true for these inputs
}

}  // namespace

extern "C" int dns_fp64_fma_rate(double seconds, double *tflops) {
    if (!tflops || !(seconds > 0.0) || seconds > 10.0) return DNS_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DNS_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return DNS_ERR_CUDA;
    const int blocks = sms * kBlocksPerSm;
    const double per_iter = 2.0 * kChains * (double)kThreads * blocks;  // flops per loop iteration
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return DNS_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return DNS_ERR_CUDA;
    }
    int rc = DNS_OK;
    long long iters = 4096;
    float ms = 0.f;
    for (int round = 0; round < 2 && rc == DNS_OK; ++round) {
        cudaEventRecord(e0, 0);
        k_dfma_rate<<<blocks, kThreads>>>(iters, 0.999999999, 1e-9);
        cudaEventRecord(e1, 0);
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f)) {
            rc = DNS_ERR_CUDA;
            break;
        }
        if (round == 0) {
            // scale the loop to the requested duration (at most 2^31 iterations)
            const double want = seconds * 1e3 / ms * (double)iters;
            iters = (long long)fmin(fmax(want, 1024.0), 2147483648.0);
        }
    }
    if (rc == DNS_OK) *tflops = per_iter * (double)iters / (ms * 1e-3) / 1e12;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}
