// The z pass (P3) with one warp per physical line: FP32, N = 16 N1 with
// N1 in {16, 32} (N = 256, 512).
//
// Per physical line (x, y) the pass takes the six spectral z lines of u and
// omega^ (fields 0..5 of B, kz <= K), transforms them to physical space,
// forms u x omega pointwise and transforms the three products back, keeping
// kz <= K (Eq. NSfinal's nonlinear term along z; Eq. ffteq's inverse and
// forward real transforms).  Pairs of real fields share one complex line:
// (ux + i uy), (uz + i wz / S), (wx + i wy) on the way in (the pairing and
// the power-of-two scale S of P3Pairs), (Nx + i Ny) and (Nz + 0 i) on the
// way out.
//
// Each length-N complex transform is a two-factor Cooley-Tukey split
// N = N1 * 16 done by one warp with a single exchange through shared memory:
//
//   inverse, x[n1 + N1 n2] = sum_k2 e^{+2 pi i k2 n2/16} e^{+2 pi i k2 n1/N}
//                              sum_k1 X[16 k1 + k2] e^{+2 pi i k1 n1/N1}
//     step I1  item k2 (16 per line): N1-point DFT over k1, twiddle
//     step I2  item n1 (N1 per line): 16-point DFT over k2
//   forward, Y[k2 + 16 k1] = sum_n1 e^{-2 pi i k1 n1/N1} e^{-2 pi i k2 n1/N}
//                              sum_n2 y[n1 + N1 n2] e^{-2 pi i k2 n2/16}
//     step F1  item n1: 16-point DFT over n2
//     step F2  item k2: twiddle, N1-point DFT over n1
//
// Step I2 leaves item n1 the physical points z = n1 + N1 n2 of all three
// packed lines, which are exactly the inputs of step F1: the cross product
// and F1 run in registers right after I2.  The exchanges I1 -> I2 and
// F1 -> F2 go through a per-warp shared-memory buffer whose rows are padded
// to an odd number of 8-byte words, so every warp access is two wavefronts
// (the minimum for 64-bit values).  The unpack of the (Nx + i Ny) line needs
// Z[k] and Z[N - k]; those sit in lanes k2 and 16 - k2 of the same half-warp
// and are exchanged by shuffles.  Only warp-level synchronisation is used.
//
// The input is read straight from HBM into registers by step I1 (a half-warp
// reads 16 consecutive kz of one field: 128-byte segments; each stored
// coefficient is read for n and for N - n, the second read from L1).  Warps
// are persistent: each walks units of LW = 32 / N1 consecutive lines with a
// stride of the grid's warp count.  The twiddles a lane needs,
// e^{-2 pi i k2 n1 / N} for its fixed k2 = lane mod 16, are factored as
// n1 = 8 a + b and held in registers: 7 + N1/8 - 1 table values per lane.
#pragma once

#include "dns_passes.cuh"

namespace dns {

template <int N> struct ZW {
    static constexpr int N1 = N / 16;
    static_assert(N1 == 16 || N1 == 32, "the warp z pass covers N = 256 and 512");
    static constexpr int LW = 32 / N1;  // lines per warp (one unit)
    static constexpr int K = GeoN<N>::K, Kzp = GeoN<N>::Kzp;
    static constexpr int P1 = 17;       // row pitch of the I1 -> I2 buffer [3 LW][N1][16 (+1)]
    static constexpr int P2 = N1 + 1;   // row pitch of the F1 -> F2 buffer [2 LW][16][N1 (+1)]
    static constexpr int BUF1 = 3 * LW * N1 * P1;
    static constexpr int BUF2 = 2 * LW * 16 * P2;
    static constexpr int WARP_CPLX = (BUF1 > BUF2 ? BUF1 : BUF2) + 1;  // + 1: keep 16-byte alignment
    static constexpr int NA = N1 / 8;
    static constexpr size_t smem(int warps) { return sizeof(float2) * (size_t)WARP_CPLX * (size_t)warps; }
};

// e^{-2 pi i k2 (8 a + b) / N} from the factors held by the lane.
template <int A, int Bf, int NA>
__device__ __forceinline__ float2 zw_twiddle(const float2 (&wa)[NA], const float2 (&wb)[8]) {
    if constexpr (A == 0 && Bf == 0) return make_float2(1.f, 0.f);
    else if constexpr (A == 0) return wb[Bf];
    else if constexpr (Bf == 0) return wa[A];
    else return cmul(wa[A], wb[Bf]);
}

template <int N, int N1, int NA, int I = 1>
__device__ __forceinline__ void zw_twiddle_all(float2 *v, const float2 (&wa)[NA], const float2 (&wb)[8], bool inverse) {
    if constexpr (I < N1) {
        float2 w = zw_twiddle<I / 8, I % 8, NA>(wa, wb);
        if (inverse) w.y = -w.y;
        v[I] = cmul(v[I], w);
        zw_twiddle_all<N, N1, NA, I + 1>(v, wa, wb, inverse);
    }
}

// Coefficient n of packed line (a + i b), Hermitian-extended along z, where
// the half-warp's 16 consecutive positions n = 16 k1 + k2 (k2 = 0..15) are
// classified at compile time: all kept, none kept, or decided per lane.
template <int N, int K1>
__device__ __forceinline__ float2 zw_load(const float2 *__restrict__ fa, const float2 *__restrict__ fb, int k2,
                                          float bscale, const Chk &ck) {
    constexpr int K = GeoN<N>::K;
    constexpr int lo = 16 * K1, hi = 16 * K1 + 15;
    // kz(n) = n for n <= N/2, N - n above; kept iff kz <= K
    constexpr bool all_low = hi <= K;
    constexpr bool all_high = lo >= N - K && lo > N / 2;
    constexpr bool none = lo > K && hi < N - K;
    if constexpr (none) {
        return make_float2(0.f, 0.f);
    } else {
        const int n = lo + k2;
        const bool low = all_low || (!all_high && n <= N / 2);
        const int kz = low ? n : N - n;
        if (!(all_low || all_high) && kz > K) return make_float2(0.f, 0.f);
        float2 a = DNS_LD(ck, fa + kz), b = DNS_LD(ck, fb + kz);
        if (K1 == 0 && n == 0) {  // Im of X[0] is ignored by the real inverse
            a.y = 0.f;
            b.y = 0.f;
        }
        b.x *= bscale;
        b.y *= bscale;
        return low ? make_float2(a.x - b.y, a.y + b.x) : make_float2(a.x + b.y, b.x - a.y);
    }
}

template <int N, int N1, int K1 = 0>
__device__ __forceinline__ void zw_load_all(float2 *v, const float2 *fa, const float2 *fb, int k2, float bscale,
                                            const Chk &ck) {
    if constexpr (K1 < N1) {
        v[K1] = zw_load<N, K1>(fa, fb, k2, bscale, ck);
        zw_load_all<N, N1, K1 + 1>(v, fa, fb, k2, bscale, ck);
    }
}

// Stores of the forward outputs k = k2 + 16 k1 (kz <= K): line f = 0 is
// Nx + i Ny (unpacked with Z[N - k] from the partner lane), f = 1 is Nz.
template <int N, int N1, int K1 = 0>
__device__ __forceinline__ void zw_store_all(const float2 *v, int k2, int lane, int f, float2 *__restrict__ dst,
                                             long long sB, const Chk &ck) {
    constexpr int K = GeoN<N>::K;
    if constexpr (16 * K1 <= K) {
        // Z[N - k]: k2 > 0 -> lane 16 - k2 of this half-warp, entry N1 - 1 - K1;
        //           k2 = 0 -> this lane, entry (N1 - K1) mod N1
        const int src = (lane & 16) | ((16 - k2) & 15);
        float2 zm;
        zm.x = __shfl_sync(0xffffffffu, v[N1 - 1 - K1].x, src);
        zm.y = __shfl_sync(0xffffffffu, v[N1 - 1 - K1].y, src);
        if (k2 == 0) zm = v[(N1 - K1) % N1];
        const int kz = k2 + 16 * K1;
        if (kz <= K) {
            const float2 za = v[K1];
            if (f == 0) {
                DNS_ST(ck, dst + kz, make_float2(0.5f * (za.x + zm.x), 0.5f * (za.y - zm.y)));
                DNS_ST(ck, dst + sB + kz, make_float2(0.5f * (za.y + zm.y), -0.5f * (za.x - zm.x)));
            } else {
                DNS_ST(ck, dst + 2 * sB + kz, za);
            }
        }
        zw_store_all<N, N1, K1 + 1>(v, k2, lane, f, dst, sB, ck);
    }
}

template <int N, int WPB, int MINB>
__global__ void __launch_bounds__(32 * WPB, MINB) k_p3_zwarp(Geo g, const float2 *__restrict__ twg,
                                                              float2 *__restrict__ B, long long nunits) {
    typedef ZW<N> Z;
    constexpr int N1 = Z::N1, LW = Z::LW, NA = Z::NA, P1 = Z::P1, P2 = Z::P2;
    constexpr long long sB = GeoN<N>::sB, NN = (long long)N * N;
    constexpr int Kzp = Z::Kzp;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float2 *buf = reinterpret_cast<float2 *>(smem_raw) + warp * Z::WARP_CPLX;
    const int k2 = lane & 15;
    float2 wb[8], wa[NA];
    wb[0] = make_float2(1.f, 0.f);
    wa[0] = make_float2(1.f, 0.f);
#pragma unroll
    for (int b = 1; b < 8; ++b) wb[b] = DNS_LD(g, twg + (k2 * b) % N);
#pragma unroll
    for (int a = 1; a < NA; ++a) wa[a] = DNS_LD(g, twg + (8 * k2 * a) % N);

    const long long nw = (long long)gridDim.x * WPB;
    for (long long u = (long long)blockIdx.x * WPB + warp; u < nunits; u += nw) {
        const long long line0 = u * LW;  // LW divides N * N: a unit never straddles two boxes
        float2 *Bb = B + (line0 / NN) * GeoN<N>::bB + (line0 % NN) * Kzp;

        // ---- I1: item (p, line, k2) of the 3 LW packed lines
        constexpr int ITEMS1 = 3 * LW * 16, ROUNDS1 = (ITEMS1 + 31) / 32;
#pragma unroll 1
        for (int r = 0; r < ROUNDS1; ++r) {
            const int item = r * 32 + lane;
            if (ITEMS1 % 32 == 0 || item < ITEMS1) {
                const int pl = item >> 4, p = pl / LW, ln = pl % LW;
                const float2 *fa = Bb + P3Pairs<N>::fa(p) * sB + ln * Kzp;
                const float2 *fb = Bb + P3Pairs<N>::fb(p) * sB + ln * Kzp;
                float2 v[N1];
                zw_load_all<N, N1>(v, fa, fb, k2, p == 1 ? (float)(1.0 / P3Pairs<N>::S) : 1.f, g.chk());
                dft<N1, +1>(v);
                zw_twiddle_all<N, N1, NA>(v, wa, wb, true);
                float2 *dst = buf + pl * N1 * P1 + k2;
#pragma unroll
                for (int n1 = 0; n1 < N1; ++n1) dst[n1 * P1] = v[n1];
            }
        }
        __syncwarp();

        // ---- I2 + cross product + F1: item n1 of line ln (one item per lane)
        {
            const int ln = lane / N1, n1 = lane % N1;
            float2 x0[16], x1[16], x2[16];
            const float2 *s0 = buf + ((0 * LW + ln) * N1 + n1) * P1;
            const float2 *s1 = buf + ((1 * LW + ln) * N1 + n1) * P1;
            const float2 *s2 = buf + ((2 * LW + ln) * N1 + n1) * P1;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                x0[j] = s0[j];
                x1[j] = s1[j];
                x2[j] = s2[j];
            }
            dft<16, +1>(x0);
            dft<16, +1>(x1);
            dft<16, +1>(x2);
            // point z = n1 + N1 j: (ux, uy), (uz, wz / S), (wx, wy)
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float ux = x0[j].x, uy = x0[j].y, uz = x1[j].x, wz = x1[j].y * (float)P3Pairs<N>::S,
                            wx = x2[j].x, wy = x2[j].y;
                x0[j] = make_float2(uy * wz - uz * wy, uz * wx - ux * wz);
                x1[j] = make_float2(ux * wy - uy * wx, 0.f);
            }
            dft<16, -1>(x0);
            dft<16, -1>(x1);
            __syncwarp();  // every lane has read the I1 buffer before it is reused
            float2 *d0 = buf + ((0 * LW + ln) * 16) * P2 + n1;
            float2 *d1 = buf + ((1 * LW + ln) * 16) * P2 + n1;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                d0[j * P2] = x0[j];
                d1[j * P2] = x1[j];
            }
        }
        __syncwarp();

        // ---- F2 + unpack: item (f, line, k2); LW = 1: f = lane / 16 in one
        // round; LW = 2: round f, line = lane / 16
#pragma unroll 1
        for (int r = 0; r < LW; ++r) {
            const int f = LW == 1 ? (lane >> 4) : r;
            const int ln = LW == 1 ? 0 : (lane >> 4);
            const float2 *src = buf + ((f * LW + ln) * 16 + k2) * P2;
            float2 v[N1];
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) v[n1] = src[n1];
            zw_twiddle_all<N, N1, NA>(v, wa, wb, false);
            dft<N1, -1>(v);
            zw_store_all<N, N1>(v, k2, lane, f, Bb + ln * Kzp, sB, g.chk());
        }
        __syncwarp();  // the buffer is free for the next unit
    }
}

}  // namespace dns
