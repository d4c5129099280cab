// Kinetic energy and dissipation of a spectral field without any device
// allocation (dns_energy_noalloc in include/dns.h).
//
// Some callers cannot allocate device memory at the point where they need
// these diagnostics: callbacks and real-time loops that must not enter the
// allocator (a device allocation can synchronise the device or block), or
// processes whose device memory is a fixed budget or pool owned by another
// framework.  This entry point
// keeps its scratch (one pair of partial sums per kx plane) in a file-scope
// device array, so it allocates nothing and needs no handle.
//
// The array is shared by every call on a device and keeps the last call's
// contents.  Each call writes every slot it later reads (one block per kx
// plane writes its own pair, the final block reads only those), so nothing
// has to start at zero; calls that overlap on the GPU (on different streams,
// or from several host threads) race on the array and must be serialised by
// the caller.
#include "dns.h"

#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#define DNS_NOALLOC_MAX_N 1024
#define DNS_NOALLOC_MAX_DEVICES 64

namespace {

// partial sums: [2 * kx + 0] = sum w |uhat|^2, [2 * kx + 1] = sum w |k|^2 |uhat|^2;
// the last two slots hold (E, eps) on their way to a host output
static __device__ __align__(256) double g_noalloc_scratch[2 * DNS_NOALLOC_MAX_N + 2];

double *g_scratch_addr[DNS_NOALLOC_MAX_DEVICES] = {};
std::mutex g_setup_mutex;

// One block per kx plane of a full-layout field uhat[3][N][N][N/2+1]; weights
// w = 1 on the kz = 0 and kz = N/2 planes, 2 elsewhere (half-spectrum Parseval).
template <typename C>
__global__ void k_plane_sums(int N, const C *__restrict__ uhat, double *__restrict__ scratch) {
    const int ix = blockIdx.x, Nh = N / 2 + 1;
    const long long plane = (long long)N * Nh, field = (long long)N * plane;
    const double kx = ix <= N / 2 ? ix : ix - N;
    double se = 0.0, sd = 0.0;
    for (long long e = threadIdx.x; e < plane; e += blockDim.x) {
        const int kz = (int)(e % Nh), iy = (int)(e / Nh);
        const double ky = iy <= N / 2 ? iy : iy - N;
        const long long m = (long long)ix * plane + e;
        double p = 0.0;
        for (int c = 0; c < 3; ++c) {
            const C v = uhat[c * field + m];
            p += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
        }
        const double w = (kz == 0 || 2 * kz == N) ? 1.0 : 2.0;
        se += w * p;
        sd += w * (kx * kx + ky * ky + (double)kz * kz) * p;
    }
    __shared__ double rs[2][32];
    for (int o = 16; o > 0; o >>= 1) {
        se += __shfl_down_sync(0xffffffffu, se, o);
        sd += __shfl_down_sync(0xffffffffu, sd, o);
    }
    if ((threadIdx.x & 31) == 0) {
        rs[0][threadIdx.x >> 5] = se;
        rs[1][threadIdx.x >> 5] = sd;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += rs[0][w];
            b += rs[1][w];
        }
        scratch[2 * ix] = a;
        scratch[2 * ix + 1] = b;
    }
}

// Adds the N pairs in a fixed order: out[0] = E, out[1] = eps.
__global__ void k_finish(int N, double nu, const double *__restrict__ scratch, double *__restrict__ out) {
    if (threadIdx.x != 0) return;
    double a = 0.0, b = 0.0;
    for (int ix = 0; ix < N; ++ix) {
        a += scratch[2 * ix];
        b += scratch[2 * ix + 1];
    }
    const double N3 = (double)N * N * N;
    out[0] = a / (2.0 * N3 * N3);
    out[1] = nu * b / (N3 * N3);
}

// The device address of g_noalloc_scratch on the current device, looked up
// once per device (a host-side reference to the array is not a device address).
cudaError_t scratch_for_current_device(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= DNS_NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        double *p = nullptr;
        e = cudaGetSymbolAddress((void **)&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int dns_energy_noalloc(int N, int dtype, const void *uhat, double nu, double *out, int out_on_device,
                                  void *cuda_stream) {
    if (!uhat || !out || dtype < DNS_F32 || dtype > DNS_F32_ACC64 || !std::isfinite(nu) || nu < 0.0)
        return DNS_ERR_ARG;
    if (N < 2 || (N & 1)) return DNS_ERR_ARG;
    if (N > DNS_NOALLOC_MAX_N) return DNS_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    double *scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) return DNS_ERR_CUDA;
    // the two results go to the caller's device buffer, or to the two last
    // slots of the array and then to the caller's host buffer
    if (dtype == DNS_F32)
        k_plane_sums<float2><<<N, 256, 0, st>>>(N, (const float2 *)uhat, scratch);
    else
        k_plane_sums<double2><<<N, 256, 0, st>>>(N, (const double2 *)uhat, scratch);
    if (cudaGetLastError() != cudaSuccess) return DNS_ERR_CUDA;
    if (out_on_device) {
        k_finish<<<1, 32, 0, st>>>(N, nu, scratch, out);
        if (cudaGetLastError() != cudaSuccess) return DNS_ERR_CUDA;
        return DNS_OK;
    }
    double *res = scratch + 2 * DNS_NOALLOC_MAX_N;
    k_finish<<<1, 32, 0, st>>>(N, nu, scratch, res);
    if (cudaGetLastError() != cudaSuccess) return DNS_ERR_CUDA;
    if (cudaMemcpyAsync(out, res, 2 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess) return DNS_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return DNS_ERR_CUDA;
    if (!std::isfinite(out[0]) || !std::isfinite(out[1])) return DNS_ERR_NONFINITE;
    return DNS_OK;
}
