// Building blocks of the learned subgrid closure for a coarse LES on top of
// the pseudo-spectral solver (not in the paper): a complex 3D FFT on full
// arrays, the sharp-cutoff filter that moves a DNS field to the LES mesh,
// the filtered velocity gradients and subgrid stresses, and the closure
// term -i k_j tau_ij^ added to the LES right-hand side.
//
// Full complex arrays are [F][N][N][N] (z fastest, FFT order on every axis);
// real fields travel as complex with zero imaginary part.  Sizes are small
// (the LES mesh, or the DNS mesh when building training data), so plain
// complex transforms keep this code short.
#pragma once

#include "dns_passes.cuh"

namespace dns {
namespace les {

// ---------------------------------------------------------------- complex 3D FFT
// Axis 0 (x) and 1 (y): column tiles of W consecutive z lines; axis 2 (z):
// contiguous lines, L per block (row engine).  In place; SIGN = -1 forward,
// +1 inverse (unscaled).
template <int N, int W, int T, int SIGN, int AXIS>
__global__ void __launch_bounds__(T) k_c2c_axis(float2 *__restrict__ a, const float2 *__restrict__ twg) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *tw = reinterpret_cast<float2 *>(smem_raw);
    float2 *tile = tw + N;
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = twg[i];
    __syncthreads();
    if constexpr (AXIS < 2) {
        const int z0 = blockIdx.x * W, other = blockIdx.y, f = blockIdx.z;
        const long long N3 = (long long)N * N * N;
        // axis 0: rows x at stride N*N, block fixes y; axis 1: rows y at stride N, block fixes x
        const long long stride = AXIS == 0 ? (long long)N * N : N;
        float2 *base = a + f * N3 + (AXIS == 0 ? (long long)other * N : (long long)other * N * N) + z0;
        auto load = [&](int n, int c) -> float2 { return base[n * stride + c]; };
        auto store = [&](int n, int c, float2 v) { base[n * stride + c] = v; };
        TileFFT<float, N, W, T, SIGN, 16>::run(tile, W, tw, load, store);
    } else {
        constexpr int L = W;
        float2 *base = a + (long long)blockIdx.x * L * N;
        auto load = [&](int vl, int n) -> float2 { return base[(long long)vl * N + n]; };
        auto store = [&](int vl, int n, float2 v) { base[(long long)vl * N + n] = v; };
        RowFFT<float, N, L, T, SIGN, 16>::run(tile, tw, load, store);
    }
}

// ---------------------------------------------------------------- spectral helpers
__device__ __forceinline__ int fft_k(int i, int N) { return i <= N / 2 ? i : i - N; }

// compact state (3 fields, mesh geometry g) -> full complex arrays:
//   mode 0: out[c] = uhat_c (c < 3);   mode 1: out[3i+j] = i k_j uhat_i (9 fields)
// scaled by `scale`; kz < 0 comes from Hermitian symmetry, modes outside the
// stored set are zero.
__global__ void k_compact_to_full_c(Geo g, const float2 *__restrict__ U, float2 *__restrict__ out, int mode,
                                    float scale) {
    const int N = g.N, K = g.K;
    const long long N3 = (long long)N * N * N;
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int nf = mode == 0 ? 3 : 9;
    if (e >= nf * N3) return;
    const int f = (int)(e / N3);
    const long long p = e % N3;
    const int iz = (int)(p % N), iy = (int)((p / N) % N), ix = (int)(p / ((long long)N * N));
    int kx = fft_k(ix, N), ky = fft_k(iy, N), kz = fft_k(iz, N);
    float2 v = make_float2(0.f, 0.f);
    const bool conj = kz < 0;
    if (conj) {
        kx = -kx;
        ky = -ky;
        kz = -kz;
    }
    if (abs(kx) <= K && abs(ky) <= K && kz <= K && !(2 * kz == N)) {
        const int cx = kx >= 0 ? kx : kx + g.Kx, cy = ky >= 0 ? ky : ky + g.Kx;
        const long long m = ((long long)cx * g.Kx + cy) * g.Kzp + kz;
        const int comp = mode == 0 ? f : f / 3;
        float2 u = U[comp * g.sS + m];
        if (mode == 1) {  // i k_j u at the stored (kx, ky, kz >= 0) representative
            const int j = f % 3;
            const float kj = (float)(j == 0 ? kx : (j == 1 ? ky : kz));
            u = make_float2(-kj * u.y, kj * u.x);
        }
        v = conj ? make_float2(u.x, -u.y) : u;
    }
    out[e] = make_float2(v.x * scale, v.y * scale);
}

// Full complex spectrum on mesh Ns -> full complex spectrum on mesh Nd,
// keeping |k_i| <= kc and multiplying by `scale` (the sharp cutoff filter).
__global__ void k_filter_full(const float2 *__restrict__ src, int Ns, float2 *__restrict__ dst, int Nd, int nfield,
                              int kc, float scale) {
    const long long N3 = (long long)Nd * Nd * Nd, S3 = (long long)Ns * Ns * Ns;
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= nfield * N3) return;
    const int f = (int)(e / N3);
    const long long p = e % N3;
    const int iz = (int)(p % Nd), iy = (int)((p / Nd) % Nd), ix = (int)(p / ((long long)Nd * Nd));
    const int kx = fft_k(ix, Nd), ky = fft_k(iy, Nd), kz = fft_k(iz, Nd);
    float2 v = make_float2(0.f, 0.f);
    if (abs(kx) <= kc && abs(ky) <= kc && abs(kz) <= kc) {
        const long long q = (((long long)((kx + Ns) % Ns) * Ns) + (ky + Ns) % Ns) * Ns + (kz + Ns) % Ns;
        const float2 s = src[f * S3 + q];
        v = make_float2(s.x * scale, s.y * scale);
    }
    dst[e] = v;
}

// Products of the real parts: out[q] = Re u[a_q] Re u[b_q] (imaginary 0),
// q = xx, yy, zz, xy, xz, yz.
__global__ void k_products(const float2 *__restrict__ u, long long N3, float2 *__restrict__ out) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= 6 * N3) return;
    const int q = (int)(e / N3);
    const long long p = e % N3;
    const int a = q < 3 ? q : (q == 5 ? 1 : 0), b = q < 3 ? q : (q == 3 ? 1 : 2);
    out[e] = make_float2(u[a * N3 + p].x * u[b * N3 + p].x, 0.f);
}

// tau_q = filt(u_a u_b) - ubar_a ubar_b at the LES points, and the real
// parts of gradient / stress arrays packed to [F][n^3] floats.
__global__ void k_tau_from_parts(const float2 *__restrict__ filt_prod, const float2 *__restrict__ ubar, long long n3,
                                 float *__restrict__ tau) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= 6 * n3) return;
    const int q = (int)(e / n3);
    const long long p = e % n3;
    const int a = q < 3 ? q : (q == 5 ? 1 : 0), b = q < 3 ? q : (q == 3 ? 1 : 2);
    tau[e] = filt_prod[e].x - ubar[a * n3 + p].x * ubar[b * n3 + p].x;
}

__global__ void k_real_part(const float2 *__restrict__ a, long long n, float *__restrict__ out, float scale) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e < n) out[e] = scale * a[e].x;
}

__global__ void k_real_to_c(const float *__restrict__ a, long long n, float2 *__restrict__ out) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e < n) out[e] = make_float2(a[e], 0.f);
}

// Smagorinsky stresses (the classic eddy-viscosity comparator, not in the
// paper): S_ij = (g_ij + g_ji)/2 with g[3i+j] = d_j u_i, |S| = sqrt(2 S_ij S_ij),
// tau_q = -2 c2 |S| S_q for q = xx, yy, zz, xy, xz, yz, c2 = (C_s Delta)^2.
__global__ void k_smagorinsky(const float *__restrict__ g, long long V, float c2, float *__restrict__ tau) {
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= V) return;
    float a[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) a[q] = g[q * V + p];
    const float sxx = a[0], syy = a[4], szz = a[8];
    const float sxy = 0.5f * (a[1] + a[3]), sxz = 0.5f * (a[2] + a[6]), syz = 0.5f * (a[5] + a[7]);
    const float ss = sxx * sxx + syy * syy + szz * szz + 2.f * (sxy * sxy + sxz * sxz + syz * syz);
    const float f = -2.f * c2 * sqrtf(2.f * ss);
    tau[p] = f * sxx;
    tau[V + p] = f * syy;
    tau[2 * V + p] = f * szz;
    tau[3 * V + p] = f * sxy;
    tau[4 * V + p] = f * sxz;
    tau[5 * V + p] = f * syz;
}

// Closure forcing on the stored modes of the LES mesh: f_i = -i k_j tau_ij^
// from the forward-transformed stresses (full complex [6][n][n][n]); the
// update pass projects it together with the nonlinear term.
__global__ void k_closure_forcing(Geo g, const float2 *__restrict__ th, float2 *__restrict__ F) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= g.sS) return;
    const int kz = (int)(e % g.Kzp);
    const long long r = e / g.Kzp;
    const int iy = (int)(r % g.Kx), ix = (int)(r / g.Kx);
    float2 f[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    if (kz < g.Kz) {
        const int N = g.N;
        const int k[3] = {compact_to_k(ix, g.K), compact_to_k(iy, g.K), kz};
        const long long N3 = (long long)N * N * N;
        const long long q = (((long long)((k[0] + N) % N) * N) + (k[1] + N) % N) * N + kz;
        const int idx[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                const float2 t = th[idx[i][j] * N3 + q];
                // -i k_j t = (k_j t.y, -k_j t.x)
                f[i].x += (float)k[j] * t.y;
                f[i].y -= (float)k[j] * t.x;
            }
    }
    F[e] = f[0];
    F[g.sS + e] = f[1];
    F[2 * g.sS + e] = f[2];
}

}  // namespace les
}  // namespace dns
