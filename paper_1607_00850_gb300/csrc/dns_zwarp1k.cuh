// The z pass (P3) with one warp per physical line at N = 1024, FP32: the
// same computation as dns_zwarp.cuh (Eq. NSfinal's nonlinear term along z,
// the packed pairs of P3Pairs, u x omega between the inverse and forward
// transforms), with the split N = 64 * 16.
//
//   inverse, x[n1 + 64 n2] = sum_k2 e^{+2 pi i k2 n2/16} e^{+2 pi i k2 n1/N}
//                              sum_k1 X[16 k1 + k2] e^{+2 pi i k1 n1/64}
//     I1  item (p, k2): 64-point DFT over k1, twiddle        48 per line
//     I2  item n1: 16-point DFT over k2 of the three lines   64 per line
//   forward, Y[k2 + 16 k1] = sum_n1 e^{-2 pi i k1 n1/64} e^{-2 pi i k2 n1/N}
//                              sum_n2 y[n1 + 64 n2] e^{-2 pi i k2 n2/16}
//     F1  item n1: u x omega, 16-point DFTs of two lines     64 per line
//     F2  item (f, k2): twiddle, 64-point DFT over n1        32 per line
//
// A 64-point transform in one lane would hold 128 registers, so every I1
// and F2 item is split over the lanes k2 and k2 + 16 (h = lane / 16): one
// radix-2 step of decimation in frequency through a shuffle (the lane of
// half h holds inputs 32 h + m, m < 32; it forms the sum (h = 0) or the
// difference times e^{-+2 pi i m/64} (h = 1)), then a 32-point DFT per lane,
// whose output r is entry 2 r + h.  I1 runs one round per packed line
// (16 items x 2 halves); F2 one round per output line.
//
// I2 and F1 take two rounds per line (n1 = 32 q + lane).  The I1 -> I2
// buffer is kept in two halves by n1 (q = 0: n1 < 32, q = 1: n1 >= 32), and
// the F1 output of round q goes into half q, which its own I2 has just read;
// the F2 lane of half h reads n1 = 32 h + m, i.e. exactly half h.  Rows are
// padded to an odd number of 8-byte words (P1 = 17, P2 = 33).
//
// All three inverse lines take the same arithmetic (u x omega's z component
// is Im(conj(U) W), whose box mean cancels the rounding shared by the U and
// W lines).  The unpack of (Nx + i Ny) takes Z[N - k] from lane
// (16 - k2) + 16 (1 - h), entry 31 - r (k2 > 0), or from its own lane
// (k2 = 0).  Twiddles: per lane, the factors of n1 = 16 a + (2 b + h)
// (inverse, I1) and of n1 = 32 h + 8 a + b (forward, F2), 11 table values
// each, one product per twiddle.
#pragma once

#include "dns_zwarp.cuh"

namespace dns {

struct ZW1k {
    static constexpr int N = 1024, N1 = 64;
    static constexpr int K = GeoN<N>::K, Kzp = GeoN<N>::Kzp;
    static constexpr int P1 = 17, P2 = 33;
    static constexpr int HALF = 3 * 32 * P1;  // one half of the I1 -> I2 buffer [3][32][17]
    static_assert(2 * 16 * P2 <= HALF, "a half holds its F1 output [2][16][33]");
    static constexpr int WARP_CPLX = 2 * HALF;  // even: every warp's buffer stays 16-byte aligned
    static constexpr size_t smem(int warps) { return sizeof(float2) * (size_t)WARP_CPLX * (size_t)warps; }
};

// cos(2 pi m / 64), m = 0..16; the rest by symmetry
__host__ __device__ constexpr double kCos64(int m) {
    return m == 0 ? 1.0
         : m == 1 ? 0.9951847266721968862448
         : m == 2 ? 0.9807852804032304491262
         : m == 3 ? 0.9569403357322088649358
         : m == 4 ? 0.9238795325112867561282
         : m == 5 ? 0.8819212643483550297128
         : m == 6 ? 0.8314696123025452370788
         : m == 7 ? 0.7730104533627369608109
         : m == 8 ? 0.7071067811865475244008
         : m == 9 ? 0.6343932841636454982152
         : m == 10 ? 0.5555702330196022247428
         : m == 11 ? 0.4713967368259976485564
         : m == 12 ? 0.3826834323650897717285
         : m == 13 ? 0.2902846772544623676362
         : m == 14 ? 0.1950903220161282678483
         : m == 15 ? 0.0980171403295606019942
         : 0.0;
}
// e^{+2 pi i m / 64}, 0 <= m < 32, as (cos, sin)
__host__ __device__ constexpr double w64_re(int m) { return m <= 16 ? kCos64(m) : -kCos64(32 - m); }
__host__ __device__ constexpr double w64_im(int m) { return m <= 16 ? kCos64(16 - m) : kCos64(m - 16); }

template <int K0, int CNT, int M = 0>
__device__ __forceinline__ void zw1k_load(float2 *v, const float2 *fa, const float2 *fb, int k2, float bscale,
                                          const Chk &ck) {
    if constexpr (M < CNT) {
        v[M] = zw_load<1024, K0 + M>(fa, fb, k2, bscale, ck);
        zw1k_load<K0, CNT, M + 1>(v, fa, fb, k2, bscale, ck);
    }
}

// The radix-2 step of a 64-point transform split over lanes k2, k2 + 16:
// a[m] holds input 32 h + m; on return, the 32-point inputs of half h.
// SIGN = +1 inverse, -1 forward.
template <int SIGN>
__device__ __forceinline__ void zw1k_split(float2 *a, int h) {
    const float sg = h ? -1.f : 1.f;
#pragma unroll
    for (int m = 0; m < 32; ++m) {
        float2 b;
        b.x = __shfl_xor_sync(0xffffffffu, a[m].x, 16);
        b.y = __shfl_xor_sync(0xffffffffu, a[m].y, 16);
        a[m] = make_float2(fmaf(sg, a[m].x, b.x), fmaf(sg, a[m].y, b.y));
    }
    if (h) {
#pragma unroll
        for (int m = 1; m < 32; ++m) {
            const float2 w = make_float2((float)w64_re(m), (float)(SIGN * w64_im(m)));
            a[m] = cmul(a[m], w);
        }
    }
}

// Outputs of F2's line f for this lane's entries k1 = 2 r + h (kz <= K),
// with the (Nx + i Ny) unpack for f = 0.
template <int R = 0>
__device__ __forceinline__ void zw1k_store(const float2 *v, int k2, int h, int f, float2 *__restrict__ dst,
                                           long long sB, const Chk &ck) {
    constexpr int K = ZW1k::K;
    if constexpr (32 * R <= K) {  // entry 2R + h holds kz >= 32 R
        const int src = ((16 - k2) & 15) | ((1 - h) << 4);
        float2 zm;
        zm.x = __shfl_sync(0xffffffffu, v[31 - R].x, src);
        zm.y = __shfl_sync(0xffffffffu, v[31 - R].y, src);
        if (k2 == 0) zm = h ? v[31 - R] : v[(32 - R) & 31];
        const int kz = k2 + 16 * (2 * R + h);
        if (kz <= K) {
            const float2 za = v[R];
            if (f == 0) {
                DNS_ST(ck, dst + kz, make_float2(0.5f * (za.x + zm.x), 0.5f * (za.y - zm.y)));
                DNS_ST(ck, dst + sB + kz, make_float2(0.5f * (za.y + zm.y), -0.5f * (za.x - zm.x)));
            } else {
                DNS_ST(ck, dst + 2 * sB + kz, za);
            }
        }
        zw1k_store<R + 1>(v, k2, h, f, dst, sB, ck);
    }
}

template <int WPB, int MINB>
__global__ void __launch_bounds__(32 * WPB, MINB) k_p3_zwarp1k(Geo g, const float2 *__restrict__ twg,
                                                                float2 *__restrict__ B, long long nunits) {
    typedef ZW1k Z;
    constexpr int N = Z::N, P1 = Z::P1, P2 = Z::P2, HALF = Z::HALF, Kzp = Z::Kzp;
    constexpr long long sB = GeoN<N>::sB, NN = (long long)N * N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float2 *buf = reinterpret_cast<float2 *>(smem_raw) + warp * Z::WARP_CPLX;
    const int k2 = lane & 15, h = lane >> 4;
    const Chk ck = g.chk();
    // I1 twiddles e^{-2 pi i k2 n1/N} (conjugated at use), n1 = 16 a + 2 b + h
    float2 ib[8], ia[4];
    // F2 twiddles e^{-2 pi i k2 n1/N}, n1 = 32 h + 8 a + b
    float2 fb[8], fa[4];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        ib[b] = DNS_LD(ck, twg + (k2 * (2 * b + h)) % N);
        fb[b] = DNS_LD(ck, twg + (k2 * (32 * h + b)) % N);
    }
    ia[0] = fa[0] = make_float2(1.f, 0.f);
#pragma unroll
    for (int a = 1; a < 4; ++a) {
        ia[a] = DNS_LD(ck, twg + (16 * k2 * a) % N);
        fa[a] = DNS_LD(ck, twg + (8 * k2 * a) % N);
    }

    const long long nw = (long long)gridDim.x * WPB;
    for (long long u = (long long)blockIdx.x * WPB + warp; u < nunits; u += nw) {
        float2 *Bb = B + (u / NN) * GeoN<N>::bB + (u % NN) * Kzp;

        // ---- I1: round p = packed line p, lane (k2, h)
#pragma unroll 1
        for (int p = 0; p < 3; ++p) {
            const float2 *fa0 = Bb + P3Pairs<N>::fa(p) * sB;
            const float2 *fb0 = Bb + P3Pairs<N>::fb(p) * sB;
            const float bs = p == 1 ? (float)(1.0 / P3Pairs<N>::S) : 1.f;
            float2 a[32];
            if (h == 0) zw1k_load<0, 32>(a, fa0, fb0, k2, bs, ck);
            else zw1k_load<32, 32>(a, fa0, fb0, k2, bs, ck);
            zw1k_split<+1>(a, h);
            dft<32, +1>(a);
            // entry r is n1 = 2 r + h = 16 a + 2 b + h (r = 8 a + b); its
            // row in half q = n1 / 32 = r / 16
#pragma unroll
            for (int r = 0; r < 32; ++r) {
                const int ai = r / 8, bi = r % 8;
                float2 w = ai == 0 ? ib[bi] : cmul(ia[ai], ib[bi]);
                w.y = -w.y;
                const float2 y = (r == 0 && h == 0) ? a[r] : cmul(a[r], w);
                const int n1l = (2 * r + h) & 31, q = r >> 4;
                buf[q * HALF + (p * 32 + n1l) * P1 + k2] = y;
            }
        }
        __syncwarp();

        // ---- I2 + cross product + F1: two rounds of 32 items n1 = 32 q + lane
#pragma unroll 1
        for (int q = 0; q < 2; ++q) {
            float2 *hb = buf + q * HALF;
            float2 x0[16], x1[16], x2[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                x0[j] = hb[(0 * 32 + lane) * P1 + j];
                x1[j] = hb[(1 * 32 + lane) * P1 + j];
                x2[j] = hb[(2 * 32 + lane) * P1 + j];
            }
            dft<16, +1>(x0);
            dft<16, +1>(x1);
            dft<16, +1>(x2);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float ux = x0[j].x, uy = x0[j].y, uz = x1[j].x, wz = x1[j].y * (float)P3Pairs<N>::S,
                            wx = x2[j].x, wy = x2[j].y;
                x0[j] = make_float2(uy * wz - uz * wy, uz * wx - ux * wz);
                x1[j] = make_float2(ux * wy - uy * wx, 0.f);
            }
            dft<16, -1>(x0);
            dft<16, -1>(x1);
            __syncwarp();  // every lane has read this half before its F1 output overwrites it
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                hb[(0 * 16 + j) * P2 + lane] = x0[j];
                hb[(1 * 16 + j) * P2 + lane] = x1[j];
            }
        }
        __syncwarp();

        // ---- F2: round f = output line f, lane (k2, h) holds n1 = 32 h + m
#pragma unroll 1
        for (int f = 0; f < 2; ++f) {
            const float2 *src = buf + h * HALF + (f * 16 + k2) * P2;
            float2 v[32];
#pragma unroll
            for (int m = 0; m < 32; ++m) {
                const int ai = m / 8, bi = m % 8;
                const float2 w = ai == 0 ? fb[bi] : cmul(fa[ai], fb[bi]);
                v[m] = (m == 0 && h == 0) ? src[m] : cmul(src[m], w);
            }
            zw1k_split<-1>(v, h);
            dft<32, -1>(v);
            zw1k_store(v, k2, h, f, Bb, sB, ck);
        }
        __syncwarp();  // the buffer is free for the next unit
    }
}

}  // namespace dns
