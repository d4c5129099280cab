// Launch shapes and host launchers for one mesh size N.  Compiled once per
// supported N (dns_inst.cu with -DDNS_N=...), so the kernel units build in
// parallel.
#pragma once

#include "dns_internal.h"
#include "dns_passes.cuh"

namespace dns {

// Launch shapes.  Column passes use 128-byte tile rows (16 complex floats or
// 8 complex doubles); P3 packs L lines of 3 field pairs.  BUD = register
// budget per thread and stage (32 complex floats or 16 complex doubles),
// which fixes the thread count; RC / R3 cap the radix of the column passes
// and of P3 (larger radices mean fewer shared-memory round trips).
template <typename real, int N> struct Shape {
    static constexpr bool f32 = sizeof(real) == 4;
    static constexpr int BUD = f32 ? 32 : 16;
    static constexpr int RC = f32 ? 16 : 8;
    static constexpr int R3 = f32 ? 32 : 16;
    static constexpr int W = f32 ? 16 : 8;
    static constexpr int T = tile_threads(N, W, BUD);
    static constexpr int pow2 = (N & -N);  // largest power of two dividing N
    static constexpr int L3w = f32 ? (N >= 768 ? 4 : 8) : (N >= 768 ? 2 : 4);
    static constexpr int L3 = L3w < pow2 ? L3w : pow2;
    static constexpr int T3 = tile_threads(N, 3 * L3, BUD);
    static constexpr int LZ = L3;  // physical-input z pass
    static constexpr int TZ = tile_threads(N, 2 * LZ, BUD);
    typedef typename CT<real>::t cplx;
    static constexpr size_t smem_col = sizeof(cplx) * (size_t)(N + N * W);
    static constexpr size_t smem_p3 = sizeof(cplx) * (size_t)(N + 3 * L3 * row_ld(N));
    static constexpr size_t smem_zf = sizeof(cplx) * (size_t)(N + N * (2 * LZ + 1));
};

template <typename K> static cudaError_t set_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

static inline int cdiv(int a, int b) { return (a + b - 1) / b; }

template <typename real, int N> struct ColLaunch {
    typedef Shape<real, N> S;
    typedef typename CT<real>::t cplx;

    static cudaError_t p1(const Geo &g, const void *tw, const void *U, const void *Om, void *A, double scale,
                          cudaStream_t st) {
        auto k = k_p1_xinv<real, N, S::W, S::T, S::RC>;
        dim3 grid(6 * g.nb, cdiv(g.Kz, S::W), g.Kx);
        k<<<grid, S::T, S::smem_col, st>>>(g, (const cplx *)tw, (const cplx *)U, (const cplx *)Om, (cplx *)A,
                                           (real)scale);
        return cudaGetLastError();
    }
    static cudaError_t curl(const Geo &g, const void *U, void *Om, cudaStream_t st) {
        const long long n = g.sS * g.nb;
        k_curl<real><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, (const cplx *)U, (cplx *)Om);
        return cudaGetLastError();
    }
    static cudaError_t p5a(const Geo &g, const void *tw, const void *A, void *Nh, cudaStream_t st) {
        auto k = k_p5a_xfwd<real, N, S::W, S::T, S::RC>;
        dim3 grid(3 * g.nb, cdiv(g.Kz, S::W), g.Kx);
        k<<<grid, S::T, S::smem_col, st>>>(g, (const cplx *)tw, (const cplx *)A, (cplx *)Nh);
        return cudaGetLastError();
    }
    static cudaError_t p2(const Geo &g, const void *tw, const void *A, void *B, cudaStream_t st) {
        auto k = k_p2_yinv<real, N, S::W, S::T, S::RC>;
        dim3 grid(cdiv(g.Kz, S::W), N, 6 * g.nb);
        k<<<grid, S::T, S::smem_col, st>>>(g, (const cplx *)tw, (const cplx *)A, (cplx *)B);
        return cudaGetLastError();
    }
    static cudaError_t p3(const Geo &g, const void *tw, void *B, cudaStream_t st) {
        auto k = k_p3_z_cross<real, N, S::L3, S::T3, S::R3>;
        dim3 grid((unsigned)((long long)N * N / S::L3 * g.nb));
        k<<<grid, S::T3, S::smem_p3, st>>>(g, (const cplx *)tw, (cplx *)B);
        return cudaGetLastError();
    }
    static cudaError_t p4(const Geo &g, const void *tw, const void *B, void *A, cudaStream_t st) {
        auto k = k_p4_yfwd<real, N, S::W, S::T, S::RC>;
        dim3 grid(cdiv(g.Kz, S::W), N, 3 * g.nb);
        k<<<grid, S::T, S::smem_col, st>>>(g, (const cplx *)tw, (const cplx *)B, (cplx *)A);
        return cudaGetLastError();
    }
    template <typename ioreal>
    static cudaError_t zfwd(const Geo &g, const void *tw, const void *u, void *B, cudaStream_t st) {
        auto k = k_zfwd_real<real, ioreal, N, S::LZ, S::TZ, S::R3>;
        dim3 grid((unsigned)((long long)N * N / S::LZ));
        k<<<grid, S::TZ, S::smem_zf, st>>>(g, (const cplx *)tw, (const ioreal *)u, (cplx *)B);
        return cudaGetLastError();
    }
};

template <typename real, typename acc> struct UpdLaunch {
    typedef typename CT<real>::t cplx;
    typedef typename CT<acc>::t cacc;
    static cudaError_t p5b(const Geo &g, const void *Nh, const UpdateArgsErased &e, cudaStream_t st) {
        UpdateArgs<real, acc> a;
        a.U = (const cplx *)e.U;
        a.U0 = (const cacc *)e.U0;
        a.U1 = (cacc *)e.U1;
        a.Uout = (cplx *)e.Uout;
        a.U0out = (cacc *)e.U0out;
        a.dU = (cacc *)e.dU;
        a.Om = (cplx *)e.Om;
        a.nu = e.nu;
        a.nu_box = e.nu_box;
        a.adt = e.adt;
        a.bdt = e.bdt;
        a.stage = e.stage;
        const long long n = g.sS * g.nb;
        const unsigned blocks = (unsigned)((n + 255) / 256);
        k_p5b_update<real, acc><<<blocks, 256, 0, st>>>(g, (const cplx *)Nh, a);
        return cudaGetLastError();
    }
};

// Raise the dynamic shared-memory limit of every kernel of one (N, dtype);
// called once at handle creation, outside any stream capture.
template <typename real, typename ioreal, int N> cudaError_t prepare_all() {
    typedef Shape<real, N> S;
    cudaError_t e;
    if ((e = set_smem(k_p1_xinv<real, N, S::W, S::T, S::RC>, S::smem_col)) != cudaSuccess) return e;
    if ((e = set_smem(k_p2_yinv<real, N, S::W, S::T, S::RC>, S::smem_col)) != cudaSuccess) return e;
    if ((e = set_smem(k_p3_z_cross<real, N, S::L3, S::T3, S::R3>, S::smem_p3)) != cudaSuccess) return e;
    if ((e = set_smem(k_p4_yfwd<real, N, S::W, S::T, S::RC>, S::smem_col)) != cudaSuccess) return e;
    if ((e = set_smem(k_zfwd_real<real, ioreal, N, S::LZ, S::TZ, S::R3>, S::smem_zf)) != cudaSuccess) return e;
    return set_smem(k_p5a_xfwd<real, N, S::W, S::T, S::RC>, S::smem_col);
}

template <int N> bool fill_passes(int dtype, PassSet *ps) {
    if (dtype == 1) {
        typedef Shape<double, N> S;
        ps->W = S::W; ps->T = S::T; ps->L3 = S::L3; ps->T3 = S::T3;
        ps->smem_col = S::smem_col; ps->smem_p3 = S::smem_p3;
        ps->p1 = ColLaunch<double, N>::p1;
        ps->curl = ColLaunch<double, N>::curl;
        ps->p2 = ColLaunch<double, N>::p2;
        ps->p3 = ColLaunch<double, N>::p3;
        ps->p4 = ColLaunch<double, N>::p4;
        ps->p5a = ColLaunch<double, N>::p5a;
        ps->p5b = UpdLaunch<double, double>::p5b;
        ps->zfwd = ColLaunch<double, N>::template zfwd<double>;
        ps->prepare = prepare_all<double, double, N>;
        return true;
    }
    if (dtype == 0 || dtype == 2) {
        typedef Shape<float, N> S;
        ps->W = S::W; ps->T = S::T; ps->L3 = S::L3; ps->T3 = S::T3;
        ps->smem_col = S::smem_col; ps->smem_p3 = S::smem_p3;
        ps->p1 = ColLaunch<float, N>::p1;
        ps->curl = ColLaunch<float, N>::curl;
        ps->p2 = ColLaunch<float, N>::p2;
        ps->p3 = ColLaunch<float, N>::p3;
        ps->p4 = ColLaunch<float, N>::p4;
        ps->p5a = ColLaunch<float, N>::p5a;
        if (dtype == 0) {
            ps->p5b = UpdLaunch<float, float>::p5b;
            ps->zfwd = ColLaunch<float, N>::template zfwd<float>;
            ps->prepare = prepare_all<float, float, N>;
        } else {
            ps->p5b = UpdLaunch<float, double>::p5b;
            ps->zfwd = ColLaunch<float, N>::template zfwd<double>;
            ps->prepare = prepare_all<float, double, N>;
        }
        return true;
    }
    return false;
}

}  // namespace dns
