// Launch shapes and host launchers for one mesh size N.  Compiled once per
// supported N (dns_inst.cu with -DDNS_N=...), so the kernel units build in
// parallel.
//
// Every tuned pass is compiled in a few shapes ("variants"); the autotuner
// times them on the device and picks one per pass (variant 0 is the default).
//   column passes (P1, P2, P4, P5a): W lines per tile x radix cap RC
//   z pass (P3):                      L lines per block x radix cap R3
// The thread count follows from a register budget per thread and stage (BUD:
// 32 complex floats or 16 complex doubles): T = W N / BUD rounded up to 32.
// Shapes whose threads exceed 1024 or whose shared memory exceeds the 227 KB
// a block may use are not compiled; meshes below 64 compile only variant 0.
#pragma once

#include "dns_internal.h"
#include "dns_passes.cuh"
#include "dns_zwarp.cuh"
#include "dns_zwarp1k.cuh"

namespace dns {

constexpr size_t kMaxSmem = 227 * 1024;

template <typename real> struct VariantTable;
// P3 variants: lines per block lmax >> p3S (lmax = the most lines that fit
// 512 threads), radix cap p3R, blocks the compiler keeps resident p3M, and
// how the input arrives and is processed, p3A: 0 loads by the threads, 1
// persistent blocks fed by bulk asynchronous copies (next group
// prefetched), 2 one group per block by one bulk copy into the tile, 3 as 2
// with the inverse-last / cross / forward-first stages fused in registers.
template <> struct VariantTable<float> {
    static constexpr int BUD = 32;
    static constexpr int colW[5] = {16, 32, 16, 16, 8};
    static constexpr int colR[5] = {16, 16, 8, 32, 32};
    static constexpr int p3S[14] = {0, 0, 1, 1, 2, 0, 0, 1, 0, 0, 1, 0, 1, 1};
    static constexpr int p3R[14] = {32, 32, 32, 32, 32, 16, 32, 32, 32, 32, 32, 32, 32, 32};
    static constexpr int p3M[14] = {1, 2, 1, 2, 2, 1, 1, 2, 1, 2, 2, 1, 1, 2};
    static constexpr int p3A[14] = {0, 0, 0, 0, 0, 0, 1, 1, 2, 2, 2, 3, 3, 3};
};
template <> struct VariantTable<double> {
    static constexpr int BUD = 16;
    static constexpr int colW[5] = {8, 16, 8, 8, 4};
    static constexpr int colR[5] = {8, 8, 16, 32, 32};
    static constexpr int p3S[14] = {0, 0, 1, 1, 2, 0, 0, 1, 0, 0, 1, 0, 1, 1};
    static constexpr int p3R[14] = {16, 16, 16, 16, 16, 8, 16, 16, 16, 16, 16, 16, 16, 16};
    static constexpr int p3M[14] = {1, 2, 1, 2, 2, 1, 1, 2, 1, 2, 2, 1, 1, 2};
    static constexpr int p3A[14] = {0, 0, 0, 0, 0, 0, 1, 1, 2, 2, 2, 3, 3, 3};
};

__host__ __device__ constexpr int raw_threads(int N, int W, int BUD) {
    return (((N * W + BUD - 1) / BUD + 31) / 32) * 32;
}
__host__ __device__ constexpr int at_least_32(int t) { return t < 32 ? 32 : t; }

// Column variants 0..3 load their input with the threads; 4..7 are the same
// shapes fed by bulk copies of the tile's input rows; 8 and 9 are the half-
// width shape (64-byte rows: a third of the shared memory of 128-byte rows
// at 1024^3, so three blocks share an SM where one did) loaded by the
// threads and by bulk copies.
template <typename real, int N, int V> struct ColShape {
    typedef VariantTable<real> VT;
    static constexpr int SH = V < 8 ? V % 4 : 4;
    static constexpr int W = VT::colW[SH];
    static constexpr int RC = VT::colR[SH];
    static constexpr bool BULK = V < 8 ? V >= 4 : V == 9;
    static constexpr int T = at_least_32(raw_threads(N, W, VT::BUD));
    typedef typename CT<real>::t cplx;
    static constexpr size_t smem = sizeof(cplx) * (size_t)(N + N * W);
    static constexpr bool valid = (V == 0 || N >= 64) && T <= 1024 && smem <= kMaxSmem;
};

__host__ __device__ constexpr int pow2_floor(int x) {
    int p = 1;
    while (2 * p <= x) p *= 2;
    return p;
}

// P3 keeps at most 512 threads per block (at least 128 registers each) and
// at most 16 lines; lmax is the largest such power of two dividing N.
template <typename real, int N, int V> struct P3Shape {
    typedef VariantTable<real> VT;
    static constexpr int pow2 = (N & -N);  // largest power of two dividing N
    static constexpr int lfit = pow2_floor(512 * VT::BUD / (3 * N)) < 1 ? 1 : pow2_floor(512 * VT::BUD / (3 * N));
    static constexpr int lmax = lfit < 16 ? (lfit < pow2 ? lfit : pow2) : (16 < pow2 ? 16 : pow2);
    static constexpr int L = (lmax >> VT::p3S[V]) < 1 ? 1 : (lmax >> VT::p3S[V]);
    static constexpr int R3 = VT::p3R[V];
    static constexpr int T = at_least_32(raw_threads(N, 3 * L, VT::BUD));
    typedef typename CT<real>::t cplx;
    static constexpr bool ASYNC = VT::p3A[V] == 1;
    static constexpr bool BULK = VT::p3A[V] == 2;
    static constexpr bool BULKF = VT::p3A[V] == 3;
    static constexpr size_t smem =
        ASYNC ? P3Stage<real, N, L, R3>::smem
              : sizeof(cplx) * (size_t)(N + twt_size(N, R3) + (BULKF ? twt_size(N, R3, true) : 0) + 3 * L * row_ld(N));
    static constexpr int MINB = VT::p3M[V];
    static constexpr bool valid = (V == 0 || (N >= 64 && (lmax >> VT::p3S[V]) >= 1)) && T <= 1024 &&
                                  smem <= kMaxSmem && (MINB == 1 || (2 * smem <= kMaxSmem && 2 * T <= 1024));
};

// physical-input z pass (column-mapped, not tuned)
template <typename real, int N> struct ZShape {
    typedef VariantTable<real> VT;
    static constexpr int pow2 = (N & -N);
    static constexpr int Lw = sizeof(real) == 4 ? 8 : 4;
    static constexpr int LZ = Lw < pow2 ? Lw : pow2;
    static constexpr int T = at_least_32(raw_threads(N, 2 * LZ, VT::BUD));
    static constexpr int R = sizeof(real) == 4 ? 32 : 16;
    typedef typename CT<real>::t cplx;
    static constexpr size_t smem = sizeof(cplx) * (size_t)(N + N * (2 * LZ + 1));
};

template <typename K> static cudaError_t set_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

static inline int cdiv(int a, int b) { return (a + b - 1) / b; }

template <typename real, int N, int V> struct ColLaunch {
    typedef ColShape<real, N, V> S;
    typedef typename CT<real>::t cplx;
    static cudaError_t p1(const Geo &g, const void *tw, const void *U, const void *Om, void *A, double scale,
                          cudaStream_t st) {
        dim3 grid(6 * g.nb, cdiv(g.Kz, S::W), g.Kx);
        k_p1_xinv<real, N, S::W, S::T, S::RC, S::BULK><<<grid, S::T, S::smem, st>>>(
            g, (const cplx *)tw, (const cplx *)U, (const cplx *)Om, (cplx *)A, (real)scale);
        return cudaGetLastError();
    }
    static cudaError_t p2(const Geo &g, const void *tw, const void *A, void *B, cudaStream_t st) {
        dim3 grid(cdiv(g.Kz, S::W), N, 6 * g.nb);
        k_p2_yinv<real, N, S::W, S::T, S::RC, S::BULK><<<grid, S::T, S::smem, st>>>(g, (const cplx *)tw, (const cplx *)A,
                                                                           (cplx *)B);
        return cudaGetLastError();
    }
    static cudaError_t p4(const Geo &g, const void *tw, const void *B, void *A, cudaStream_t st) {
        dim3 grid(cdiv(g.Kz, S::W), N, 3 * g.nb);
        k_p4_yfwd<real, N, S::W, S::T, S::RC, S::BULK><<<grid, S::T, S::smem, st>>>(g, (const cplx *)tw, (const cplx *)B,
                                                                           (cplx *)A);
        return cudaGetLastError();
    }
    static cudaError_t p5a(const Geo &g, const void *tw, const void *A, void *Nh, cudaStream_t st) {
        dim3 grid(3 * g.nb, cdiv(g.Kz, S::W), g.Kx);
        k_p5a_xfwd<real, N, S::W, S::T, S::RC, S::BULK><<<grid, S::T, S::smem, st>>>(g, (const cplx *)tw,
                                                                            (const cplx *)A, (cplx *)Nh);
        return cudaGetLastError();
    }
    static cudaError_t prepare() {
        cudaError_t e;
        if ((e = set_smem(k_p1_xinv<real, N, S::W, S::T, S::RC, S::BULK>, S::smem)) != cudaSuccess) return e;
        if ((e = set_smem(k_p2_yinv<real, N, S::W, S::T, S::RC, S::BULK>, S::smem)) != cudaSuccess) return e;
        if ((e = set_smem(k_p4_yfwd<real, N, S::W, S::T, S::RC, S::BULK>, S::smem)) != cudaSuccess) return e;
        return set_smem(k_p5a_xfwd<real, N, S::W, S::T, S::RC, S::BULK>, S::smem);
    }
};

template <typename real, int N, int V> struct P3Launch {
    typedef P3Shape<real, N, V> S;
    typedef typename CT<real>::t cplx;
    typedef void (*TmaKernel)(Geo, const cplx *, cplx *, long long);
    static inline int resident = 0;  // persistent grid: SMs x blocks per SM (set by prepare)
    static TmaKernel tma_kernel() {
        if constexpr (S::MINB == 2) return k_p3_z_tma_2b<real, N, S::L, S::T, S::R3>;
        else return k_p3_z_tma<real, N, S::L, S::T, S::R3>;
    }
    typedef void (*BulkKernel)(Geo, const cplx *, cplx *);
    static BulkKernel bulk_kernel() {
        if constexpr (S::BULKF) {
            if constexpr (S::MINB == 2) return k_p3_z_bulkf_2b<real, N, S::L, S::T, S::R3>;
            else return k_p3_z_bulkf<real, N, S::L, S::T, S::R3>;
        } else {
            if constexpr (S::MINB == 2) return k_p3_z_bulk_2b<real, N, S::L, S::T, S::R3>;
            else return k_p3_z_bulk<real, N, S::L, S::T, S::R3>;
        }
    }
    static cudaError_t p3(const Geo &g, const void *tw, void *B, cudaStream_t st) {
        if constexpr (S::ASYNC) {
            // bulk copies need 16-byte aligned rows of the stated padding
            if (g.Kzp != P3Stage<real, N, S::L>::KZP || ((uintptr_t)B & 15) || resident < 1)
                return cudaErrorInvalidValue;
            const long long groups = (long long)N * N / S::L * g.nb;
            const unsigned grid = (unsigned)(groups < resident ? groups : resident);
            tma_kernel()<<<grid, S::T, S::smem, st>>>(g, (const cplx *)tw, (cplx *)B, groups);
        } else if constexpr (S::BULK || S::BULKF) {
            if (g.Kzp != P3Stage<real, N, S::L>::KZP || ((uintptr_t)B & 15)) return cudaErrorInvalidValue;
            dim3 grid((unsigned)((long long)N * N / S::L * g.nb));
            bulk_kernel()<<<grid, S::T, S::smem, st>>>(g, (const cplx *)tw, (cplx *)B);
        } else {
            dim3 grid((unsigned)((long long)N * N / S::L * g.nb));
            if constexpr (S::MINB == 2)
                k_p3_z_cross_2b<real, N, S::L, S::T, S::R3><<<grid, S::T, S::smem, st>>>(g, (const cplx *)tw,
                                                                                       (cplx *)B);
            else
                k_p3_z_cross<real, N, S::L, S::T, S::R3><<<grid, S::T, S::smem, st>>>(g, (const cplx *)tw,
                                                                                    (cplx *)B);
        }
        return cudaGetLastError();
    }
    static cudaError_t prepare() {
        if constexpr (S::ASYNC) {
            cudaError_t e = set_smem(tma_kernel(), S::smem);
            int dev = 0, sms = 0, occ = 0;
            if (e == cudaSuccess) e = cudaGetDevice(&dev);
            if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, tma_kernel(), S::T, S::smem);
            if (e == cudaSuccess) resident = sms * (occ > 0 ? occ : 1);
            return e;
        } else if constexpr (S::BULK || S::BULKF) {
            return set_smem(bulk_kernel(), S::smem);
        } else if constexpr (S::MINB == 2) {
            return set_smem(k_p3_z_cross_2b<real, N, S::L, S::T, S::R3>, S::smem);
        } else {
            return set_smem(k_p3_z_cross<real, N, S::L, S::T, S::R3>, S::smem);
        }
    }
};

template <typename real, int N> struct MiscLaunch {
    typedef ZShape<real, N> Z;
    typedef typename CT<real>::t cplx;
    template <typename ioreal>
    static cudaError_t zfwd(const Geo &g, const void *tw, const void *u, void *B, cudaStream_t st) {
        dim3 grid((unsigned)((long long)N * N / Z::LZ));
        k_zfwd_real<real, ioreal, N, Z::LZ, Z::T, Z::R><<<grid, Z::T, Z::smem, st>>>(g, (const cplx *)tw,
                                                                                   (const ioreal *)u, (cplx *)B);
        return cudaGetLastError();
    }
    template <typename ioreal> static cudaError_t prepare() {
        return set_smem(k_zfwd_real<real, ioreal, N, Z::LZ, Z::T, Z::R>, Z::smem);
    }
    static cudaError_t curl(const Geo &g, const void *U, void *Om, cudaStream_t st) {
        const long long n = g.sS * g.nb;
        k_curl<real><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, (const cplx *)U, (cplx *)Om);
        return cudaGetLastError();
    }
};

template <typename real, typename acc> struct UpdLaunch {
    typedef typename CT<real>::t cplx;
    typedef typename CT<acc>::t cacc;
    static UpdateArgs<real, acc> args(const UpdateArgsErased &e) {
        UpdateArgs<real, acc> a;
        a.U = (const cplx *)e.U;
        a.U0 = (const cacc *)e.U0;
        a.U1 = (cacc *)e.U1;
        a.Uout = (cplx *)e.Uout;
        a.U0out = (cacc *)e.U0out;
        a.dU = (cacc *)e.dU;
        a.Om = (cplx *)e.Om;
        a.Fext = (const cplx *)e.Fext;
        a.nu = e.nu;
        a.nu_box = e.nu_box;
        a.adt = e.adt;
        a.bdt = e.bdt;
        a.stage = e.stage;
        a.dt = e.dt;
        a.ifrk = e.ifrk;
        a.rng = nullptr;
        a.err = nullptr;
        return a;
    }
    // the same with the context's range table and status word (checked accesses)
    static UpdateArgs<real, acc> args(const UpdateArgsErased &e, const Geo &g) {
        UpdateArgs<real, acc> a = args(e);
        a.rng = g.rng;
        a.err = g.err;
        return a;
    }
};

// The update pass of one mesh size (its index arithmetic uses N's geometry).
template <typename real, typename acc, int N> struct UpdLaunchN {
    typedef typename CT<real>::t cplx;
    static cudaError_t p5b(const Geo &g, const void *Nh, const UpdateArgsErased &e, cudaStream_t st) {
        static_assert(GeoN<N>::sS < (1ll << 31), "one field's stored modes index with int");
        if (g.nb < 1 || g.nb > 65535) return cudaErrorInvalidValue;
        const dim3 grid((unsigned)((GeoN<N>::sS + 255) / 256), (unsigned)g.nb);
        k_p5b_update<real, acc, N><<<grid, 256, 0, st>>>((const cplx *)Nh, UpdLaunch<real, acc>::args(e, g));
        return cudaGetLastError();
    }
};

// Fused x-forward + update (P5a + P5b): W columns of each of the three
// fields per block, radix cap RC.
template <typename real> struct FusedTable;
// BUD: complex values a thread holds per stage (sets the thread count).
template <> struct FusedTable<float> {
    static constexpr int W[2] = {8, 8};
    static constexpr int R[2] = {16, 16};
    static constexpr int BUD[2] = {32, 16};
};
template <> struct FusedTable<double> {
    static constexpr int W[2] = {4, 4};
    static constexpr int R[2] = {8, 8};
    static constexpr int BUD[2] = {16, 8};
};

template <typename real, int N, int V> struct FusedShape {
    static constexpr int W = FusedTable<real>::W[V];
    static constexpr int RC = FusedTable<real>::R[V];
    static constexpr int T = at_least_32(raw_threads(N, 3 * W, FusedTable<real>::BUD[V]));
    typedef typename CT<real>::t cplx;
    static constexpr size_t smem = sizeof(cplx) * (size_t)(N + 3 * N * W);
    static constexpr bool valid = N >= 64 && T <= 1024 && smem <= kMaxSmem;
};

template <typename real, typename acc, int N, int V> struct FusedLaunch {
    typedef FusedShape<real, N, V> S;
    typedef typename CT<real>::t cplx;
    static cudaError_t p5f(const Geo &g, const void *tw, const void *A, const UpdateArgsErased &e, cudaStream_t st) {
        dim3 grid(g.nb, cdiv(g.Kz, S::W), g.Kx);
        k_p5_fused<real, acc, N, S::W, S::T, S::RC><<<grid, S::T, S::smem, st>>>(
            g, (const cplx *)tw, (const cplx *)A, UpdLaunch<real, acc>::args(e, g));
        return cudaGetLastError();
    }
    static cudaError_t prepare() { return set_smem(k_p5_fused<real, acc, N, S::W, S::T, S::RC>, S::smem); }
};

// ------------------------------------------------------------------ tables
template <typename real, int N, int V> static void fill_col(PassSet *ps) {
    if constexpr (V < PassSet::NCOLV) {
        typedef ColShape<real, N, V> S;
        if constexpr (S::valid) {
            ps->p1[V] = ColLaunch<real, N, V>::p1;
            ps->p2[V] = ColLaunch<real, N, V>::p2;
            ps->p4[V] = ColLaunch<real, N, V>::p4;
            ps->p5a[V] = ColLaunch<real, N, V>::p5a;
            ps->prep_col[V] = ColLaunch<real, N, V>::prepare;
            ps->col_w[V] = S::W;
            ps->col_r[V] = S::RC;
            ps->col_t[V] = S::T;
        }
        fill_col<real, N, V + 1>(ps);
    }
}

// Warp-per-line z pass (dns_zwarp.cuh, N = 256 and 512; dns_zwarp1k.cuh,
// N = 1024): FP32, persistent blocks of WPB warps, in the last two P3
// variant slots.  At 256 and 512 they differ in the register cap (MINB
// blocks resident per SM); at 1024 (26 KB of shared memory per warp, so at
// most 8 warps per SM) in the block size: 4 warps x 2 blocks or 8 x 1.
template <int N, int V> struct ZWShape {
    static constexpr bool K1024 = N == 1024;
    static constexpr int WPB = K1024 ? (V == PassSet::NP3V - 2 ? 4 : 8) : 4;
    static constexpr int MINB = K1024 ? (V == PassSet::NP3V - 2 ? 2 : 1) : (V == PassSet::NP3V - 2 ? 4 : 3);
    static constexpr int T = 32 * WPB;
    static constexpr bool valid = (N == 256 || N == 512 || N == 1024);
    static constexpr int LW = K1024 ? 1 : ZW<(K1024 ? 512 : N)>::LW;   // lines per warp unit
    static constexpr int N1 = K1024 ? 64 : N / 16;
    static constexpr size_t SMEM = K1024 ? ZW1k::smem(WPB) : ZW<(K1024 ? 512 : N)>::smem(WPB);
};

template <int N, int V> struct ZWLaunch {
    typedef ZWShape<N, V> S;
    static inline int resident = 0;  // persistent grid: SMs x blocks per SM (set by prepare)
    static auto kernel() {
        if constexpr (N == 1024) return k_p3_zwarp1k<S::WPB, S::MINB>;
        else return k_p3_zwarp<N, S::WPB, S::MINB>;
    }
    static cudaError_t p3(const Geo &g, const void *tw, void *B, cudaStream_t st) {
        if (g.Kzp != GeoN<N>::Kzp || resident < 1 || g.nb < 1) return cudaErrorInvalidValue;
        const long long units = (long long)N * N / S::LW * g.nb;
        const long long blocks = (units + S::WPB - 1) / S::WPB;
        const unsigned grid = (unsigned)(blocks < resident ? blocks : resident);
        kernel()<<<grid, S::T, S::SMEM, st>>>(g, (const float2 *)tw, (float2 *)B, units);
        return cudaGetLastError();
    }
    static cudaError_t prepare() {
        cudaError_t e = set_smem(kernel(), S::SMEM);
        int dev = 0, sms = 0, occ = 0;
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel(), S::T, S::SMEM);
        if (e == cudaSuccess) resident = sms * (occ > 0 ? occ : 1);
        return e;
    }
};

template <typename real, int N, int V> static void fill_p3(PassSet *ps) {
    if constexpr (V >= PassSet::NP3V - 2 && V < PassSet::NP3V) {
        if constexpr (sizeof(real) == 4 && ZWShape<N, V>::valid) {
            ps->p3[V] = ZWLaunch<N, V>::p3;
            ps->prep_p3[V] = ZWLaunch<N, V>::prepare;
            ps->p3_l[V] = ZWShape<N, V>::LW;
            ps->p3_r[V] = ZWShape<N, V>::N1;
            ps->p3_t[V] = ZWShape<N, V>::T;
        }
        fill_p3<real, N, V + 1>(ps);
    } else if constexpr (V < PassSet::NP3V) {
        typedef P3Shape<real, N, V> S;
        if constexpr (S::valid) {
            ps->p3[V] = P3Launch<real, N, V>::p3;
            ps->prep_p3[V] = P3Launch<real, N, V>::prepare;
            ps->p3_l[V] = S::L;
            ps->p3_r[V] = S::R3;
            ps->p3_t[V] = S::T;
        }
        fill_p3<real, N, V + 1>(ps);
    }
}

template <typename real, typename acc, int N, int V> static void fill_p5f(PassSet *ps) {
    if constexpr (V < PassSet::NP5F) {
        typedef FusedShape<real, N, V> S;
        if constexpr (S::valid) {
            ps->p5f[V] = FusedLaunch<real, acc, N, V>::p5f;
            ps->prep_p5f[V] = FusedLaunch<real, acc, N, V>::prepare;
            ps->p5f_w[V] = S::W;
            ps->p5f_r[V] = S::RC;
            ps->p5f_t[V] = S::T;
        }
        fill_p5f<real, acc, N, V + 1>(ps);
    }
}

template <int N> bool fill_passes(int dtype, PassSet *ps) {
    *ps = PassSet();
    if (dtype == 1) {
        fill_col<double, N, 0>(ps);
        fill_p3<double, N, 0>(ps);
        ps->curl = MiscLaunch<double, N>::curl;
        ps->p5b = UpdLaunchN<double, double, N>::p5b;
        fill_p5f<double, double, N, 0>(ps);
        ps->zfwd = MiscLaunch<double, N>::template zfwd<double>;
        ps->prep_misc = MiscLaunch<double, N>::template prepare<double>;
        return true;
    }
    if (dtype == 0 || dtype == 2) {
        fill_col<float, N, 0>(ps);
        fill_p3<float, N, 0>(ps);
        ps->curl = MiscLaunch<float, N>::curl;
        if (dtype == 0) {
            ps->p5b = UpdLaunchN<float, float, N>::p5b;
            fill_p5f<float, float, N, 0>(ps);
            ps->zfwd = MiscLaunch<float, N>::template zfwd<float>;
            ps->prep_misc = MiscLaunch<float, N>::template prepare<float>;
        } else {
            ps->p5b = UpdLaunchN<float, double, N>::p5b;
            fill_p5f<float, double, N, 0>(ps);
            ps->zfwd = MiscLaunch<float, N>::template zfwd<double>;
            ps->prep_misc = MiscLaunch<float, N>::template prepare<double>;
        }
        return true;
    }
    return false;
}

}  // namespace dns
