// The five passes of one evaluation of Eq. NSfinal, fused with their
// pointwise work (Mortensen, Sec. 2):
//
//   P1  inverse transform along x of u and omega^ = i k x uhat, 6 fields
//       (omega^ is written by the previous stage's update, or by k_curl)
//   P2  inverse transform along y, 6 fields
//   P3  inverse real transform along z of 6 fields, u x omega pointwise,
//       forward real transform along z of 3 fields (physical values never
//       leave shared memory)
//   P4  forward transform along y, 3 fields
//   P5a forward transform along x, 3 fields, stored modes only
//   P5b Leray projection, viscous term and the RK4 stage update (or the
//       bare right-hand side), streaming over the stored modes; it also
//       writes the curl of the next stage input
//
// The inverse runs x, y, z and the forward z, y, x, the reverse order as
// Eq. ffteq requires.  Storage is pruned to the 2/3-rule set: with
// K = floor((N-1)/3) only |kx|, |ky|, kz <= K are stored ("compact" index
// i = k for k >= 0, i = k + 2K+1 for k < 0).  The inverse passes read only
// those modes and the forward passes write only those modes, so the mask of
// the nonlinear term is applied by not computing what it discards.
//
// Buffers (complex, interleaved):
//   state  S[3][Kx][Ky][Kzp]   Kx = Ky = 2K+1, Kz = K+1, Kzp = Kz rounded up to 4
//   A      [6][N][Ky][Kzp]     after P1 (x physical); P4 writes its 3 fields here
//   B      [6][N][N][Kzp]      after P2 (x, y physical); P3 writes N^ into fields 0..2;
//                              P5a writes the transformed N^ here in the state layout
#pragma once

#include "dns_async.cuh"
#include "dns_fft.cuh"

namespace dns {

struct Geo {
    int N, K, Kx, Kz, Kzp;
    long long sS;  // elements per state field  = Kx*Kx*Kzp
    long long sA;  // elements per A field      = N*Kx*Kzp
    long long sB;  // elements per B field      = N*N*Kzp
    int nb;        // boxes of this size advanced together (batch), >= 1
    long long bS, bA, bB;  // elements between consecutive boxes in the state, A and B
    int *err;      // device status word: a bounded wait that gave up writes its code here
    const unsigned long long *rng;  // address ranges of the handle (index-checked builds), or nullptr
    __host__ __device__ Chk chk() const { return Chk{rng, err}; }
};

// The dealiased geometry is a function of N alone (K = floor((N - 1) / 3), the
// 2/3 rule); kernels instantiated per mesh size read it as compile-time
// constants, so their index arithmetic folds and transform stages drop the
// work on rows known to be zero on input or discarded on output.  Geo carries
// the same values at run time (dns_init builds it from this formula).
template <int N> struct GeoN {
    static constexpr int K = (N - 1) / 3, Kx = 2 * K + 1, Kz = K + 1, Kzp = (Kz + 3) / 4 * 4;
    static constexpr long long sS = (long long)Kx * Kx * Kzp, sA = (long long)N * Kx * Kzp,
                               sB = (long long)N * N * Kzp;
    static constexpr long long bS = 3 * sS, bA = 6 * sA, bB = 6 * sB;
};

// Arguments of P5b.  stage in 0..3 performs that RK4 stage; stage = -1 writes
// the right-hand side to dU instead; stage = -2 copies the transform to dU.
template <typename real, typename acc>
struct UpdateArgs {
    typedef typename CT<real>::t cplx;
    typedef typename CT<acc>::t cacc;
    const cplx *U;   // stage input (real type); may alias U0 when real == acc
    const cacc *U0;  // state at the start of the step
    cacc *U1;        // RK4 accumulator
    cplx *Uout;      // next stage input (real type), nullptr when not needed
    cacc *U0out;     // after the last stage: the new step-start state
    cacc *dU;        // stage = -1: right-hand side out
    cplx *Om;        // curl of the next stage input (stages 0..3), nullptr to skip
    const cplx *Fext;  // extra forcing on the stored modes added before the projection, or nullptr
    double nu;
    const double *nu_box;  // per-box viscosity (batched boxes), or nullptr for nu
    double adt;      // a_s * dt
    double bdt;      // b_s * dt
    double dt;       // time step (integrating-factor scheme)
    int stage;
    int ifrk;        // 1: integrating-factor RK4 (exact viscous factor), 0: classical RK4
    const unsigned long long *rng;  // address ranges of the handle (index-checked builds), or nullptr
    int *err;        // the handle's device status word
};

__device__ __forceinline__ int compact_to_k(int i, int K) { return i <= K ? i : i - (2 * K + 1); }

// Row n of a length-N line in FFT order -> compact index, or -1 if not stored.
template <int N> __device__ __forceinline__ int row_to_compact(int n, int K) {
    if (n <= K) return n;
    if (n >= N - K) return n - N + 2 * K + 1;
    return -1;
}

template <typename real> __device__ __forceinline__ void load_twiddles(typename CT<real>::t *tw,
                                                                       const typename CT<real>::t *twg,
                                                                       int N, const Chk &ck = Chk{}) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = DNS_LD(ck, twg + i);
}

// ------------------------------------------------------------------- bulk-fed column tiles
// Rows [0, nrows) of a column tile (row r: ncols complex values at
// src + r * stride, 16-byte aligned, ncols * sizeof(cplx) a multiple of 16)
// copied by the bulk copy engine to stage[r * W ...].  rows_issue is called
// by every thread (thread 0 arms the barrier, then each thread issues rows
// tid, tid + T, ...); rows_wait waits (bounded, one thread) and returns false
// after recording the timeout, in which case the block must return.
template <typename cplx, int W>
__device__ __forceinline__ void rows_issue(const Geo &g, cplx *stage, const cplx *src, long long stride, int nrows,
                                           int ncols, uint64_t *bar) {
    const uint32_t rb = (uint32_t)(ncols * sizeof(cplx));
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_arrive_expect_tx(bar, rb * (uint32_t)nrows);
    }
    __syncthreads();
    // a row outside the handle's buffers (checked builds) is not copied; the
    // block's bounded wait then gives up
    for (int r = threadIdx.x; r < nrows; r += blockDim.x)
        if (DNS_RANGE_OK(g, src + r * stride, rb)) bulk_copy_g2s(stage + r * W, src + r * stride, rb, bar);
}

__device__ __forceinline__ bool rows_wait(uint64_t *bar, int *s_ok, int *err) {
    if (threadIdx.x == 0) *s_ok = mbar_wait_bounded(bar, 0) ? 1 : 0;
    __syncthreads();
    if (!*s_ok) {
        if (threadIdx.x == 0) {
            record_error(err, kErrWaitTimeout);
            mbar_wait_bounded(bar, 0);  // let the copies in flight land before the block ends
        }
        return false;
    }
    mbar_try_wait(bar, 0);  // completed: acquire the copied data in every thread
    return true;
}

// ------------------------------------------------------------------- P1
// Inverse transform along x of u (fields 0..2, from U) and of omega^ = i k x
// uhat (fields 3..5, from Om, written by the previous update or by k_curl).
// BULK: the Kx input rows of the tile arrive by bulk copy into the tile
// itself (the first stage reads all its inputs before its barrier).
template <typename real, int N, int W, int T, int MAXR, bool BULK>
__global__ void __launch_bounds__(T) k_p1_xinv(Geo g, const typename CT<real>::t *__restrict__ twg,
                                               const typename CT<real>::t *__restrict__ U,
                                               const typename CT<real>::t *__restrict__ Om,
                                               typename CT<real>::t *__restrict__ A, real scale) {
    typedef typename CT<real>::t cplx;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_ok;
    cplx *tw = reinterpret_cast<cplx *>(smem_raw);
    cplx *tile = tw + N;
    const int box = blockIdx.x / 6, f = blockIdx.x % 6, kz0 = blockIdx.y * W, jy = blockIdx.z;
    constexpr int K = GeoN<N>::K, Kx = GeoN<N>::Kx, Kz = GeoN<N>::Kz, Kzp = GeoN<N>::Kzp;
    const cplx *src = (f < 3 ? U + f * GeoN<N>::sS : Om + (f - 3) * GeoN<N>::sS) + box * GeoN<N>::bS + (long long)jy * Kzp;
    cplx *dst = A + box * GeoN<N>::bA + f * GeoN<N>::sA + (long long)jy * Kzp;
    if constexpr (BULK) rows_issue<cplx, W>(g, tile, src + kz0, (long long)Kx * Kzp, Kx, min(W, Kzp - kz0), &bar);
    load_twiddles<real>(tw, twg, N, g.chk());
    if constexpr (BULK) {
        if (!rows_wait(&bar, &s_ok, g.err)) return;
    } else {
        __syncthreads();
    }
    auto load = [&](int n, int c) -> cplx {
        const int kz = kz0 + c;
        const int ix = row_to_compact<N>(n, K);
        if (kz >= Kz || ix < 0) return cmk<cplx>(0.0, 0.0);
        const cplx v = BULK ? tile[ix * W + c] : DNS_LD(g, src + (long long)ix * Kx * Kzp + kz);
        return cmk<cplx>(v.x * scale, v.y * scale);
    };
    auto store = [&](int n, int c, cplx v) {
        const int kz = kz0 + c;
        if (kz < Kz) DNS_ST(g, dst + (long long)n * Kx * Kzp + kz, v);
    };
    TileFFT<real, N, W, T, +1, MAXR>::run(tile, W, tw, load, store);
}

// omega^ = i k x uhat on the stored modes (Eq. eqNS: omega = curl u):
// (i(ky w - kz v), i(kz u - kx w), i(kx v - ky u)).
template <typename cplx, typename real>
__device__ __forceinline__ void curl_mode(real kx, real ky, real kz, cplx u, cplx v, cplx w, cplx &ox, cplx &oy,
                                          cplx &oz) {
    ox = cmk<cplx>(-(ky * w.y - kz * v.y), ky * w.x - kz * v.x);
    oy = cmk<cplx>(-(kz * u.y - kx * w.y), kz * u.x - kx * w.x);
    oz = cmk<cplx>(-(kx * v.y - ky * u.y), kx * v.x - ky * u.x);
}

template <typename real>
__global__ void k_curl(Geo g, const typename CT<real>::t *__restrict__ U, typename CT<real>::t *__restrict__ Om) {
    typedef typename CT<real>::t cplx;
    const long long sS = g.sS;
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= sS * g.nb) return;
    const long long box = e / sS, mm = e % sS;
    const int kz = (int)(mm % g.Kzp);
    const long long r = mm / g.Kzp;
    const int iy = (int)(r % g.Kx), ix = (int)(r / g.Kx);
    const long long m = box * g.bS + mm;
    if (kz >= g.Kz) {
        const cplx z = cmk<cplx>(0.0, 0.0);
        DNS_ST(g, Om + m, z);
        DNS_ST(g, Om + sS + m, z);
        DNS_ST(g, Om + 2 * sS + m, z);
        return;
    }
    cplx ox, oy, oz;
    curl_mode<cplx, real>((real)compact_to_k(ix, g.K), (real)compact_to_k(iy, g.K), (real)kz, DNS_LD(g, U + m),
                          DNS_LD(g, U + sS + m), DNS_LD(g, U + 2 * sS + m), ox, oy, oz);
    DNS_ST(g, Om + m, ox);
    DNS_ST(g, Om + sS + m, oy);
    DNS_ST(g, Om + 2 * sS + m, oz);
}

// ------------------------------------------------------------------- P2
template <typename real, int N, int W, int T, int MAXR, bool BULK>
__global__ void __launch_bounds__(T) k_p2_yinv(Geo g, const typename CT<real>::t *__restrict__ twg,
                                               const typename CT<real>::t *__restrict__ A,
                                               typename CT<real>::t *__restrict__ B) {
    typedef typename CT<real>::t cplx;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_ok;
    cplx *tw = reinterpret_cast<cplx *>(smem_raw);
    cplx *tile = tw + N;
    const int kz0 = blockIdx.x * W, x = blockIdx.y, box = blockIdx.z / 6, f = blockIdx.z % 6;
    constexpr int K = GeoN<N>::K, Kx = GeoN<N>::Kx, Kz = GeoN<N>::Kz, Kzp = GeoN<N>::Kzp;
    const cplx *src = A + box * GeoN<N>::bA + f * GeoN<N>::sA + (long long)x * Kx * Kzp;
    cplx *dst = B + box * GeoN<N>::bB + f * GeoN<N>::sB + (long long)x * N * Kzp;
    if constexpr (BULK) rows_issue<cplx, W>(g, tile, src + kz0, Kzp, Kx, min(W, Kzp - kz0), &bar);
    load_twiddles<real>(tw, twg, N, g.chk());
    if constexpr (BULK) {
        if (!rows_wait(&bar, &s_ok, g.err)) return;
    } else {
        __syncthreads();
    }
    auto load = [&](int n, int c) -> cplx {
        const int kz = kz0 + c;
        const int iy = row_to_compact<N>(n, K);
        cplx z;
        z.x = 0;
        z.y = 0;
        if (kz >= Kz || iy < 0) return z;
        return BULK ? tile[iy * W + c] : DNS_LD(g, src + (long long)iy * Kzp + kz);
    };
    auto store = [&](int n, int c, cplx v) {
        const int kz = kz0 + c;
        if (kz < Kz) DNS_ST(g, dst + (long long)n * Kzp + kz, v);
    };
    TileFFT<real, N, W, T, +1, MAXR>::run(tile, W, tw, load, store);
}

// ------------------------------------------------------------------- P3
// Pairs of real fields packed into the three complex lines of the inverse
// (B fields 0..2 = u, 3..5 = omega): (ux, uy), (uz, wz), (wx, wy).  Rounding
// in a packed transform leaks a relative O(eps) part of each field of a
// pair into the other; u x omega has no product u_i w_i, so with these pairs
// the leak never forms a square (with (uz, wx), uz wx would gain
// eps (wx^2 - uz^2), a sign-definite error that adds up coherently over the
// x-y planes and shows in the (0, 0, kz) modes of the nonlinear term).  The
// mixed pair carries wz / S, S a power of two near the ratio of the two
// fields' magnitudes, so neither field's leak is amplified by |w| / |u|;
// the physical wz is multiplied back by S (both scalings are exact).
template <int N> struct P3Pairs {
    static constexpr int K = (N - 1) / 3;
    static constexpr double S = K >= 128 ? 32.0 : (K >= 32 ? 16.0 : (K >= 8 ? 8.0 : 2.0));
    static __host__ __device__ constexpr int fa(int p) { return p == 0 ? 0 : (p == 1 ? 2 : 3); }
    static __host__ __device__ constexpr int fb(int p) { return p == 0 ? 1 : (p == 1 ? 5 : 4); }
};

// L lines (consecutive y at one x) per block, row-mapped (RowFFT).  Pairs of
// real fields share one complex transform: virtual line (p, l) holds
// X_{2p} + i X_{2p+1}, extended to the full length by Hermitian symmetry
// (Z[n] = a + i b for n <= N/2, conj(a) + i conj(b) at n = N - kz); after
// the inverse transform its real and imaginary parts are the two physical
// fields.  The first inverse stage packs straight from HBM (coalesced along
// kz); the cross product is computed inside the first forward stage, so the
// physical values are read once from shared memory and never stored.
// Forward half of P3, on the tile the inverse half left in natural order
// (pair p of line l at row p*L + l): u x omega fused into the first forward
// stage (component order c0 = a1 b2 - a2 b1, c1 = a2 b0 - a0 b2,
// c2 = a0 b1 - a1 b0; line l becomes Nx + i Ny, line L + l becomes Nz + 0i),
// the remaining stages, then the two real transforms of line l unpacked and
// kz <= K stored to fields 0..2 of B (already offset to the box).
// Forward stages >= 1 of the 2L packed lines (stage 0 output in the tile),
// then the two real transforms of line l unpacked and kz <= K stored to
// fields 0..2 of B (already offset to the box).
template <typename real, int N, int L, int T, int MAXR>
__device__ __forceinline__ void p3_fwd_rest_store(const Geo &g, typename CT<real>::t *tile,
                                                  const typename CT<real>::t *tw, typename CT<real>::t *B,
                                                  long long line0) {
    typedef typename CT<real>::t cplx;
    constexpr int LDR = row_ld(N);
    constexpr int K = GeoN<N>::K, Kzp = GeoN<N>::Kzp;
    constexpr long long sB = GeoN<N>::sB;
    // the unpack below reads kz <= K of the Nz lines and kz <= K, N - kz of
    // the others: the last stage stores only those positions (K is a
    // compile-time constant, so the outputs never read are not computed)
    auto tstore = [&](int vl, int n, cplx v) {
        if (n <= K || (vl < L && n >= N - K)) tile[vl * LDR + radd(n)] = v;
    };
    auto noload = [&](int, int) -> cplx { return cmk<cplx>(0.0, 0.0); };
    constexpr FftPlan P = make_plan(N, MAXR);
    if constexpr (P.nst > 1) RowFFT<real, N, 2 * L, T, -1, MAXR, 1, false, true>::run(tile, tw, noload, tstore);
    for (int e = threadIdx.x; e < L * (K + 1); e += T) {
        const int kz = e % (K + 1), l = e / (K + 1);
        const cplx za = tile[l * LDR + radd(kz)];
        const cplx zm = tile[l * LDR + radd((N - kz) % N)];
        const cplx zb = tile[(L + l) * LDR + radd(kz)];
        const long long off = (line0 + l) * Kzp + kz;
        // X = (Z[k] + conj Z[N-k]) / 2,  Y = (Z[k] - conj Z[N-k]) / (2i)
        DNS_ST(g, B + off, cmk<cplx>(0.5 * (za.x + zm.x), 0.5 * (za.y - zm.y)));
        DNS_ST(g, B + sB + off, cmk<cplx>(0.5 * (za.y + zm.y), -0.5 * (za.x - zm.x)));
        DNS_ST(g, B + 2 * sB + off, zb);
    }
}

// The middle of P3 in registers: the last stage of the inverse (run with
// the reversed plan, so its radix R is the forward plan's first) leaves work
// item (l, j) the physical values of all three packed lines of line l at
// z = j + r N/R; u x omega of those points feeds the first forward stage
// directly, whose input positions are the same.  Saves the tile round trip
// between the two transforms.  Stage-0 forward output goes to the tile.
template <typename real, int N, int L, int T, int MAXR>
__device__ __forceinline__ void p3_mid_fused(typename CT<real>::t *tile, const typename CT<real>::t *tw) {
    typedef typename CT<real>::t cplx;
    constexpr int LDR = row_ld(N);
    constexpr FftPlan PI = make_plan_rev(N, MAXR), PF = make_plan(N, MAXR);
    constexpr int SL = PI.nst - 1;
    constexpr int R = PI.r[SL];
    static_assert(PI.nst >= 2 && R == PF.r[0], "inverse last radix must equal forward first radix");
    constexpr int NB = N / R;  // items per line; = PI.ns[SL], the last stage's twiddle period
    constexpr int TOT = NB * L;
    constexpr int Q = (TOT + T - 1) / T;
    const cplx *twl = tw + N + twt_size(N, MAXR) + twt_offset(N, MAXR, SL, true);
    cplx va[Q][R], vb[Q][R];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int idx = (int)threadIdx.x + q * T;
        if (Q * T == TOT || idx < TOT) {
            const int l = idx / NB, j = idx % NB;
            cplx x2[R], w[R];
            stage_twiddles<R>(twl + j * twt_row(R), w);
#pragma unroll
            for (int r = 1; r < R; ++r) w[r].y = -w[r].y;  // inverse transform: conjugate twiddles
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                cplx *xp = p == 0 ? va[q] : (p == 1 ? vb[q] : x2);
#pragma unroll
                for (int r = 0; r < R; ++r) xp[r] = tile[(p * L + l) * LDR + radd(j + r * NB)];
#pragma unroll
                for (int r = 1; r < R; ++r) xp[r] = cmul(xp[r], w[r]);
                dft<R, +1>(xp);
            }
            // point z = j + r NB: (ux, uy), (uz, wz / S), (wx, wy) -> Nx + i Ny, Nz + 0i
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const real ux = va[q][r].x, uy = va[q][r].y, uz = vb[q][r].x,
                           wz = vb[q][r].y * (real)P3Pairs<N>::S, wx = x2[r].x, wy = x2[r].y;
                va[q][r] = cmk<cplx>(uy * wz - uz * wy, uz * wx - ux * wz);
                vb[q][r] = cmk<cplx>(ux * wy - uy * wx, 0.0);
            }
            dft<R, -1>(va[q]);
            dft<R, -1>(vb[q]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int idx = (int)threadIdx.x + q * T;
        if (Q * T == TOT || idx < TOT) {
            const int l = idx / NB, j = idx % NB;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int a = radd(j * R + r);
                tile[l * LDR + a] = va[q][r];
                tile[(L + l) * LDR + a] = vb[q][r];
            }
        }
    }
    __syncthreads();
}

template <typename real, int N, int L, int T, int MAXR>
__device__ __forceinline__ void p3_forward_store(const Geo &g, typename CT<real>::t *tile,
                                                 const typename CT<real>::t *tw, typename CT<real>::t *B,
                                                 long long line0) {
    typedef typename CT<real>::t cplx;
    constexpr int LDR = row_ld(N);
    {
        constexpr FftPlan P = make_plan(N, MAXR);
        constexpr int R = P.r[0];
        constexpr int NB = N / R;
        constexpr int TOT = NB * L;
        constexpr int Q = (TOT + T - 1) / T;
        cplx va[Q][R], vb[Q][R];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int idx = (int)threadIdx.x + q * T;
            if (Q * T == TOT || idx < TOT) {
                const int l = idx / NB, j = idx % NB;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int a = radd(j + r * NB);
                    const cplx p0 = tile[l * LDR + a], p1 = tile[(L + l) * LDR + a], p2 = tile[(2 * L + l) * LDR + a];
                    const real ux = p0.x, uy = p0.y, uz = p1.x, wz = p1.y * (real)P3Pairs<N>::S, wx = p2.x,
                               wy = p2.y;
                    va[q][r] = cmk<cplx>(uy * wz - uz * wy, uz * wx - ux * wz);
                    vb[q][r] = cmk<cplx>(ux * wy - uy * wx, 0.0);
                }
                dft<R, -1>(va[q]);
                dft<R, -1>(vb[q]);
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int idx = (int)threadIdx.x + q * T;
            if (Q * T == TOT || idx < TOT) {
                const int l = idx / NB, j = idx % NB;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int a = radd(j * R + r);
                    tile[l * LDR + a] = va[q][r];
                    tile[(L + l) * LDR + a] = vb[q][r];
                }
            }
        }
        __syncthreads();
    }
    p3_fwd_rest_store<real, N, L, T, MAXR>(g, tile, tw, B, line0);
}

// First-stage input of the packed inverse: virtual line vl = p L + l holds
// field fa(p) + i field fb(p) of line l (fb(1) = wz divided by S),
// Hermitian-extended along z (a, b are the two fields' coefficients at
// kz = n or N - n).
template <int N, typename cplx>
__device__ __forceinline__ cplx p3_pack(cplx a, cplx b, int p, int n, int kz) {
    if (kz == 0) {
        a.y = 0;
        b.y = 0;
    }
    if (p == 1) b = cscale(b, (decltype(b.x))(1.0 / P3Pairs<N>::S));
    return n <= N / 2 ? cmk<cplx>(a.x - b.y, a.y + b.x) : cmk<cplx>(a.x + b.y, b.x - a.y);
}

template <typename real, int N, int L, int T, int MAXR>
__device__ __forceinline__ void p3_body(Geo g, const typename CT<real>::t *__restrict__ twg,
                                        typename CT<real>::t *__restrict__ B) {
    typedef typename CT<real>::t cplx;
    constexpr int LDR = row_ld(N);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx *tw = reinterpret_cast<cplx *>(smem_raw);  // N twiddles, then the per-stage tables
    cplx *tile = tw + N + twt_size(N, MAXR);         // [3L][LDR]: pair p of line l at row p*L + l
    load_twiddles<real>(tw, twg, N, g.chk());
    build_twt<cplx, N, MAXR>(tw + N, twg, g.chk());
    __syncthreads();
    constexpr int K = GeoN<N>::K, Kzp = GeoN<N>::Kzp;
    const long long lineg = (long long)blockIdx.x * L;  // = box*N*N + x*N + y0
    const long long box = lineg / ((long long)N * N), line0 = lineg % ((long long)N * N);
    constexpr long long sB = GeoN<N>::sB;
    B += box * GeoN<N>::bB;
    // ---- inverse: 3 packed lines per physical line, natural order into the tile
    auto iload = [&](int vl, int n) -> cplx {
        const int p = vl / L, l = vl % L;
        const int kz = n <= N / 2 ? n : N - n;
        if (kz > K) return cmk<cplx>(0.0, 0.0);
        const long long off = (line0 + l) * Kzp + kz;
        return p3_pack<N>(DNS_LD(g, B + P3Pairs<N>::fa(p) * sB + off), DNS_LD(g, B + P3Pairs<N>::fb(p) * sB + off), p,
                          n, kz);
    };
    auto tstore = [&](int vl, int n, cplx v) { tile[vl * LDR + radd(n)] = v; };
    RowFFT<real, N, 3 * L, T, +1, MAXR, 0, false, true>::run(tile, tw, iload, tstore);
    p3_forward_store<real, N, L, T, MAXR>(g, tile, tw, B, line0);
}

// Two launch-bound flavours of P3 (the autotuner picks): the compiler's own
// register choice, or a limit that keeps two blocks resident per SM.
template <typename real, int N, int L, int T, int MAXR>
__global__ void __launch_bounds__(T) k_p3_z_cross(Geo g, const typename CT<real>::t *__restrict__ twg,
                                                  typename CT<real>::t *__restrict__ B) {
    p3_body<real, N, L, T, MAXR>(g, twg, B);
}
template <typename real, int N, int L, int T, int MAXR>
__global__ void __launch_bounds__(T, 2) k_p3_z_cross_2b(Geo g, const typename CT<real>::t *__restrict__ twg,
                                                        typename CT<real>::t *__restrict__ B) {
    p3_body<real, N, L, T, MAXR>(g, twg, B);
}

// P3 as a persistent kernel whose line groups arrive by bulk asynchronous
// copy: each block walks groups blockIdx.x, blockIdx.x + gridDim.x, ...; the
// six input fields of a group (L consecutive lines, contiguous in B) are
// copied into a shared staging buffer, and the copy of the next group is
// issued as soon as the first inverse stage has consumed the current one, so
// it overlaps the rest of the group's transforms.  Shared memory:
// twiddles [N] and per-stage tables | tile [3L][row_ld(N)] | staging
// [6][L][Kzp] (16-byte aligned).
// A copy that does not complete within the wait limit sets g.err and ends
// the block.
template <typename real, int N, int L, int MAXR = 8> struct P3Stage {
    typedef typename CT<real>::t cplx;
    static constexpr int KZP = ((N - 1) / 3 + 1 + 3) / 4 * 4;
    static constexpr size_t head = sizeof(cplx) * (size_t)(N + twt_size(N, MAXR) + 3 * L * row_ld(N));
    static constexpr size_t off = (head + 15) / 16 * 16;
    static constexpr size_t field_bytes = sizeof(cplx) * (size_t)L * KZP;
    static constexpr size_t smem = off + 6 * field_bytes;
};

// Issue the bulk copies of group grp's six input fields (one thread).
template <typename real, int N, int L>
__device__ __forceinline__ void p3_issue(const Geo &g, const typename CT<real>::t *B, typename CT<real>::t *stage,
                                         uint64_t *bar, long long grp) {
    typedef P3Stage<real, N, L> PS;
    const long long NN = (long long)N * N, lineg = grp * L;
    const typename CT<real>::t *src = B + (lineg / NN) * GeoN<N>::bB + (lineg % NN) * PS::KZP;
    mbar_arrive_expect_tx(bar, (uint32_t)(6 * PS::field_bytes));
#pragma unroll
    for (int f = 0; f < 6; ++f)
        if (DNS_RANGE_OK(g, src + f * GeoN<N>::sB, PS::field_bytes))
            bulk_copy_g2s(stage + f * (L * PS::KZP), src + f * GeoN<N>::sB, (uint32_t)PS::field_bytes, bar);
}

// One group of L lines from the staging buffer (its copy has landed); issues
// the copy of group `next` (if >= 0) once the first stage has read the
// buffer.  Not inlined: inside the group loop the compiler would otherwise
// hoist the transforms' loop-invariant index arithmetic into registers.
template <typename real, int N, int L, int T, int MAXR>
__device__ __noinline__ void p3_tma_group(Geo g, const typename CT<real>::t *tw, typename CT<real>::t *tile,
                                          typename CT<real>::t *stage, uint64_t *bar,
                                          typename CT<real>::t *B, long long grp, long long next) {
    typedef typename CT<real>::t cplx;
    typedef P3Stage<real, N, L> PS;
    constexpr int LDR = row_ld(N);
    constexpr int K = GeoN<N>::K;
    const long long NN = (long long)N * N;
    const long long lineg = grp * L;
    const long long box = lineg / NN, line0 = lineg % NN;
    auto iload = [&](int vl, int n) -> cplx {
        const int p = vl / L, l = vl % L;
        const int kz = n <= N / 2 ? n : N - n;
        if (kz > K) return cmk<cplx>(0.0, 0.0);
        const cplx *row = stage + l * PS::KZP + kz;
        return p3_pack<N>(row[P3Pairs<N>::fa(p) * (L * PS::KZP)], row[P3Pairs<N>::fb(p) * (L * PS::KZP)], p, n, kz);
    };
    auto tstore = [&](int vl, int n, cplx v) { tile[vl * LDR + radd(n)] = v; };
    RowFFT<real, N, 3 * L, T, +1, MAXR, 0, true, true>::run(tile, tw, iload, tstore);
    // the staging buffer is free: fetch the next group while this one finishes
    if (threadIdx.x == 0 && next >= 0) {
        fence_proxy_async_smem();
        p3_issue<real, N, L>(g, B, stage, bar, next);
    }
    constexpr FftPlan P = make_plan(N, MAXR);
    if constexpr (P.nst > 1) RowFFT<real, N, 3 * L, T, +1, MAXR, 1, false, true>::run(tile, tw, iload, tstore);
    p3_forward_store<real, N, L, T, MAXR>(g, tile, tw, B + box * GeoN<N>::bB, line0);
}

template <typename real, int N, int L, int T, int MAXR>
__device__ __forceinline__ void p3_tma_body(Geo g, const typename CT<real>::t *__restrict__ twg,
                                            typename CT<real>::t *__restrict__ B, long long ngroups) {
    typedef typename CT<real>::t cplx;
    typedef P3Stage<real, N, L, MAXR> PS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_ok;
    cplx *tw = reinterpret_cast<cplx *>(smem_raw);
    cplx *tile = tw + N + twt_size(N, MAXR);
    cplx *stage = reinterpret_cast<cplx *>(smem_raw + PS::off);
    load_twiddles<real>(tw, twg, N, g.chk());
    build_twt<cplx, N, MAXR>(tw + N, twg, g.chk());
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    long long grp = blockIdx.x;
    if (threadIdx.x == 0 && grp < ngroups) p3_issue<real, N, L>(g, B, stage, &bar, grp);
    uint32_t parity = 0;
    for (; grp < ngroups; grp += gridDim.x) {
        if (threadIdx.x == 0) s_ok = mbar_wait_bounded(&bar, parity) ? 1 : 0;
        // this barrier also orders the previous group's last tile reads
        // before this group's first-stage writes
        __syncthreads();
        if (!s_ok) {
            if (threadIdx.x == 0) {
                record_error(g.err, kErrWaitTimeout);
                mbar_wait_bounded(&bar, parity);  // let the copy in flight land before the block ends
            }
            return;
        }
        mbar_try_wait(&bar, parity);  // completed: acquire the copied data in every thread
        parity ^= 1;
        const long long next = grp + gridDim.x < ngroups ? grp + gridDim.x : -1;
        p3_tma_group<real, N, L, T, MAXR>(g, tw, tile, stage, &bar, B, grp, next);
    }
}

// P3 with one group per block whose input arrives by bulk asynchronous copy
// into the tile itself (the first inverse stage reads every input value
// into registers before its barrier, so its writes may overwrite them).
// Same shared memory as k_p3_z_cross; the copy engine does the loads.
template <typename real, int N, int L, int T, int MAXR>
__device__ __forceinline__ void p3_bulk_body(Geo g, const typename CT<real>::t *__restrict__ twg,
                                             typename CT<real>::t *__restrict__ B) {
    typedef typename CT<real>::t cplx;
    typedef P3Stage<real, N, L> PS;
    constexpr int LDR = row_ld(N);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_ok;
    cplx *tw = reinterpret_cast<cplx *>(smem_raw);
    cplx *tile = tw + N + twt_size(N, MAXR);
    cplx *stage = tile;  // 16-byte aligned: an even number of complex values precede it
    const long long grp = blockIdx.x;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        p3_issue<real, N, L>(g, B, stage, &bar, grp);
    }
    load_twiddles<real>(tw, twg, N, g.chk());
    build_twt<cplx, N, MAXR>(tw + N, twg, g.chk());
    if (threadIdx.x == 0) s_ok = mbar_wait_bounded(&bar, 0) ? 1 : 0;
    __syncthreads();
    if (!s_ok) {
        if (threadIdx.x == 0) {
            record_error(g.err, kErrWaitTimeout);
            mbar_wait_bounded(&bar, 0);  // let the copy in flight land before the block ends
        }
        return;
    }
    mbar_try_wait(&bar, 0);  // completed: acquire the copied data in every thread
    constexpr int K = GeoN<N>::K;
    const long long NN = (long long)N * N, lineg = grp * L;
    const long long box = lineg / NN, line0 = lineg % NN;
    auto iload = [&](int vl, int n) -> cplx {
        const int p = vl / L, l = vl % L;
        const int kz = n <= N / 2 ? n : N - n;
        if (kz > K) return cmk<cplx>(0.0, 0.0);
        const cplx *row = stage + l * PS::KZP + kz;
        return p3_pack<N>(row[P3Pairs<N>::fa(p) * (L * PS::KZP)], row[P3Pairs<N>::fb(p) * (L * PS::KZP)], p, n, kz);
    };
    auto tstore = [&](int vl, int n, cplx v) { tile[vl * LDR + radd(n)] = v; };
    RowFFT<real, N, 3 * L, T, +1, MAXR, 0, false, true>::run(tile, tw, iload, tstore);
    p3_forward_store<real, N, L, T, MAXR>(g, tile, tw, B + box * GeoN<N>::bB, line0);
}

// Bulk-fed P3 with the register-fused middle (p3_mid_fused): shared memory
// twiddles [N] | forward tables | reversed-plan tables | tile (the staging
// buffer is the tile's start).
template <typename real, int N, int L, int T, int MAXR>
__device__ __forceinline__ void p3_bulkf_body(Geo g, const typename CT<real>::t *__restrict__ twg,
                                              typename CT<real>::t *__restrict__ B) {
    typedef typename CT<real>::t cplx;
    typedef P3Stage<real, N, L> PS;
    constexpr int LDR = row_ld(N);
    constexpr int TWTS = twt_size(N, MAXR) + twt_size(N, MAXR, true);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_ok;
    cplx *tw = reinterpret_cast<cplx *>(smem_raw);
    cplx *tile = tw + N + TWTS;
    cplx *stage = tile;  // 16-byte aligned: an even number of complex values precede it
    const long long grp = blockIdx.x;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        p3_issue<real, N, L>(g, B, stage, &bar, grp);
    }
    load_twiddles<real>(tw, twg, N, g.chk());
    build_twt<cplx, N, MAXR>(tw + N, twg, g.chk());
    build_twt<cplx, N, MAXR, true>(tw + N + twt_size(N, MAXR), twg, g.chk());
    if (threadIdx.x == 0) s_ok = mbar_wait_bounded(&bar, 0) ? 1 : 0;
    __syncthreads();
    if (!s_ok) {
        if (threadIdx.x == 0) {
            record_error(g.err, kErrWaitTimeout);
            mbar_wait_bounded(&bar, 0);  // let the copy in flight land before the block ends
        }
        return;
    }
    mbar_try_wait(&bar, 0);  // completed: acquire the copied data in every thread
    constexpr int K = GeoN<N>::K;
    const long long NN = (long long)N * N, lineg = grp * L;
    const long long box = lineg / NN, line0 = lineg % NN;
    auto iload = [&](int vl, int n) -> cplx {
        const int p = vl / L, l = vl % L;
        const int kz = n <= N / 2 ? n : N - n;
        if (kz > K) return cmk<cplx>(0.0, 0.0);
        const cplx *row = stage + l * PS::KZP + kz;
        return p3_pack<N>(row[P3Pairs<N>::fa(p) * (L * PS::KZP)], row[P3Pairs<N>::fb(p) * (L * PS::KZP)], p, n, kz);
    };
    auto tstore = [&](int vl, int n, cplx v) { tile[vl * LDR + radd(n)] = v; };
    RowFFT<real, N, 3 * L, T, +1, MAXR, 0, false, true, true, true>::run(tile, tw, iload, tstore);
    p3_mid_fused<real, N, L, T, MAXR>(tile, tw);
    p3_fwd_rest_store<real, N, L, T, MAXR>(g, tile, tw, B + box * GeoN<N>::bB, line0);
}

template <typename real, int N, int L, int T, int MAXR>
__global__ void __launch_bounds__(T) k_p3_z_bulkf(Geo g, const typename CT<real>::t *__restrict__ twg,
                                                  typename CT<real>::t *__restrict__ B) {
    p3_bulkf_body<real, N, L, T, MAXR>(g, twg, B);
}
template <typename real, int N, int L, int T, int MAXR>
__global__ void __launch_bounds__(T, 2) k_p3_z_bulkf_2b(Geo g, const typename CT<real>::t *__restrict__ twg,
                                                        typename CT<real>::t *__restrict__ B) {
    p3_bulkf_body<real, N, L, T, MAXR>(g, twg, B);
}

template <typename real, int N, int L, int T, int MAXR>
__global__ void __launch_bounds__(T) k_p3_z_bulk(Geo g, const typename CT<real>::t *__restrict__ twg,
                                                 typename CT<real>::t *__restrict__ B) {
    p3_bulk_body<real, N, L, T, MAXR>(g, twg, B);
}
template <typename real, int N, int L, int T, int MAXR>
__global__ void __launch_bounds__(T, 2) k_p3_z_bulk_2b(Geo g, const typename CT<real>::t *__restrict__ twg,
                                                       typename CT<real>::t *__restrict__ B) {
    p3_bulk_body<real, N, L, T, MAXR>(g, twg, B);
}

template <typename real, int N, int L, int T, int MAXR>
__global__ void __launch_bounds__(T) k_p3_z_tma(Geo g, const typename CT<real>::t *__restrict__ twg,
                                                typename CT<real>::t *__restrict__ B, long long ngroups) {
    p3_tma_body<real, N, L, T, MAXR>(g, twg, B, ngroups);
}
template <typename real, int N, int L, int T, int MAXR>
__global__ void __launch_bounds__(T, 2) k_p3_z_tma_2b(Geo g, const typename CT<real>::t *__restrict__ twg,
                                                      typename CT<real>::t *__restrict__ B, long long ngroups) {
    p3_tma_body<real, N, L, T, MAXR>(g, twg, B, ngroups);
}

// ------------------------------------------------------------------- physical input
// Forward real transform along z of a physical field u[3][N][N][N] (entry of
// a velocity given in physical space): lines (ux + i uy) and (uz + 0i).
template <typename real, typename ioreal, int N, int L, int T, int MAXR>
__global__ void __launch_bounds__(T) k_zfwd_real(Geo g, const typename CT<real>::t *__restrict__ twg,
                                                 const ioreal *__restrict__ u,
                                                 typename CT<real>::t *__restrict__ B) {
    typedef typename CT<real>::t cplx;
    constexpr int LD = 2 * L + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx *tw = reinterpret_cast<cplx *>(smem_raw);
    cplx *tile = tw + N;
    load_twiddles<real>(tw, twg, N, g.chk());
    constexpr int Kz = GeoN<N>::Kz, Kzp = GeoN<N>::Kzp;
    const long long line0 = (long long)blockIdx.x * L;  // one box per launch
    const long long N3 = (long long)N * N * N;
    constexpr long long sB = GeoN<N>::sB;
    for (int e = threadIdx.x; e < 2 * L * N; e += T) {
        const int z = e % N, pc = e / N, p = pc / L, c = pc % L;
        const long long off = (line0 + c) * N + z;
        if (p == 0) tile[z * LD + c] = cmk<cplx>((double)DNS_LD(g, u + off), (double)DNS_LD(g, u + N3 + off));
        else tile[z * LD + L + c] = cmk<cplx>((double)DNS_LD(g, u + 2 * N3 + off), 0.0);
    }
    __syncthreads();
    auto tload = [&](int n, int c) -> cplx { return tile[n * LD + c]; };
    auto tstore = [&](int n, int c, cplx v) { tile[n * LD + c] = v; };
    TileFFT<real, N, 2 * L, T, -1, MAXR>::run(tile, LD, tw, tload, tstore);
    for (int e = threadIdx.x; e < L * Kz; e += T) {
        const int kz = e % Kz, c = e / Kz;
        const cplx za = tile[kz * LD + c];
        const cplx zm = tile[((N - kz) % N) * LD + c];
        const cplx zb = tile[kz * LD + L + c];
        const long long off = (line0 + c) * Kzp + kz;
        DNS_ST(g, B + off, cmk<cplx>(0.5 * (za.x + zm.x), 0.5 * (za.y - zm.y)));
        DNS_ST(g, B + sB + off, cmk<cplx>(0.5 * (za.y + zm.y), -0.5 * (za.x - zm.x)));
        DNS_ST(g, B + 2 * sB + off, zb);
    }
}

// ------------------------------------------------------------------- P4
template <typename real, int N, int W, int T, int MAXR, bool BULK>
__global__ void __launch_bounds__(T) k_p4_yfwd(Geo g, const typename CT<real>::t *__restrict__ twg,
                                               const typename CT<real>::t *__restrict__ B,
                                               typename CT<real>::t *__restrict__ A) {
    typedef typename CT<real>::t cplx;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_ok;
    cplx *tw = reinterpret_cast<cplx *>(smem_raw);
    cplx *tile = tw + N;
    const int kz0 = blockIdx.x * W, x = blockIdx.y, box = blockIdx.z / 3, f = blockIdx.z % 3;
    constexpr int K = GeoN<N>::K, Kx = GeoN<N>::Kx, Kz = GeoN<N>::Kz, Kzp = GeoN<N>::Kzp;
    const cplx *src = B + box * GeoN<N>::bB + f * GeoN<N>::sB + (long long)x * N * Kzp;
    cplx *dst = A + box * GeoN<N>::bA + f * GeoN<N>::sA + (long long)x * Kx * Kzp;
    if constexpr (BULK) rows_issue<cplx, W>(g, tile, src + kz0, Kzp, N, min(W, Kzp - kz0), &bar);
    load_twiddles<real>(tw, twg, N, g.chk());
    if constexpr (BULK) {
        if (!rows_wait(&bar, &s_ok, g.err)) return;
    } else {
        __syncthreads();
    }
    auto load = [&](int n, int c) -> cplx {
        const int kz = kz0 + c;
        if (kz >= Kz) return cmk<cplx>(0.0, 0.0);
        return BULK ? tile[n * W + c] : DNS_LD(g, src + (long long)n * Kzp + kz);
    };
    auto store = [&](int n, int c, cplx v) {
        const int kz = kz0 + c;
        const int iy = row_to_compact<N>(n, K);
        if (kz < Kz && iy >= 0) DNS_ST(g, dst + (long long)iy * Kzp + kz, v);
    };
    TileFFT<real, N, W, T, -1, MAXR>::run(tile, W, tw, load, store);
}

// ------------------------------------------------------------------- P5
// Classical RK4 stage update of element e from this stage's right-hand side
// du; u0, u1 are the step-start state and the accumulator at e, loaded by
// the caller (before any store, so every load of a mode is in flight at
// once).  Returns the next stage input (field type): what the next P1
// transforms.
template <typename real, typename acc>
__device__ __forceinline__ typename CT<real>::t rk_update(const UpdateArgs<real, acc> &a, long long e,
                                                          typename CT<real>::t du, typename CT<acc>::t u0,
                                                          typename CT<acc>::t u1) {
    typedef typename CT<real>::t cplx;
    typedef typename CT<acc>::t cacc;
    if (a.stage < 0) {
        DNS_ST(a, a.dU + e, cmk<cacc>((acc)du.x, (acc)du.y));
        return du;
    }
    const acc dx = (acc)du.x, dy = (acc)du.y;
    const acc adt = (acc)a.adt, bdt = (acc)a.bdt;
    if (a.stage == 0) u1 = u0;
    u1.x += adt * dx;
    u1.y += adt * dy;
    cplx next;
    if (a.stage < 3) {
        DNS_ST(a, a.U1 + e, u1);
        next = cmk<cplx>((double)(u0.x + bdt * dx), (double)(u0.y + bdt * dy));
        DNS_ST(a, a.Uout + e, next);
    } else {
        DNS_ST(a, a.U0out + e, u1);
        next = cmk<cplx>((double)u1.x, (double)u1.y);
        if (a.Uout) DNS_ST(a, a.Uout + e, next);
    }
    return next;
}

// Integrating-factor (Lawson) RK4 stage update, k = this stage's projected
// nonlinear term (no viscous term):
//   s = 0: u1 = E2 u0 + (dt/6) E2 k,   next = E1 (u0 + dt/2 k)
//   s = 1: u1 += (dt/3) E1 k,          next = E1 u0 + dt/2 k
//   s = 2: u1 += (dt/3) E1 k,          next = E2 u0 + dt E1 k
//   s = 3: u1 += (dt/6) k  -> the new step-start state.
template <typename real, typename acc>
__device__ __forceinline__ typename CT<real>::t rk_update_if(const UpdateArgs<real, acc> &a, long long e,
                                                             typename CT<real>::t du, typename CT<acc>::t u0,
                                                             typename CT<acc>::t u1, acc e1, acc e2) {
    typedef typename CT<real>::t cplx;
    const acc dx = (acc)du.x, dy = (acc)du.y, dt = (acc)a.dt;
    cplx next;
    if (a.stage == 0) {
        const acc c = (dt / (acc)6) * e2;
        u1.x = e2 * u0.x + c * dx;
        u1.y = e2 * u0.y + c * dy;
        next = cmk<cplx>((double)(e1 * (u0.x + (dt / (acc)2) * dx)), (double)(e1 * (u0.y + (dt / (acc)2) * dy)));
    } else if (a.stage == 1) {
        const acc c = (dt / (acc)3) * e1;
        u1.x += c * dx;
        u1.y += c * dy;
        next = cmk<cplx>((double)(e1 * u0.x + (dt / (acc)2) * dx), (double)(e1 * u0.y + (dt / (acc)2) * dy));
    } else if (a.stage == 2) {
        const acc c = (dt / (acc)3) * e1;
        u1.x += c * dx;
        u1.y += c * dy;
        const acc d = dt * e1;
        next = cmk<cplx>((double)(e2 * u0.x + d * dx), (double)(e2 * u0.y + d * dy));
    } else {
        const acc c = dt / (acc)6;
        u1.x += c * dx;
        u1.y += c * dy;
        next = cmk<cplx>((double)u1.x, (double)u1.y);
    }
    if (a.stage < 3) {
        DNS_ST(a, a.U1 + e, u1);
        DNS_ST(a, a.Uout + e, next);
    } else {
        DNS_ST(a, a.U0out + e, u1);
        if (a.Uout) DNS_ST(a, a.Uout + e, next);
    }
    return next;
}

// P5a: forward transform along x of the 3 fields, keep the Kx stored rows;
// the result N^ (dealiased by construction) goes to a compact buffer.
template <typename real, int N, int W, int T, int MAXR, bool BULK>
__global__ void __launch_bounds__(T) k_p5a_xfwd(Geo g, const typename CT<real>::t *__restrict__ twg,
                                                const typename CT<real>::t *__restrict__ A,
                                                typename CT<real>::t *__restrict__ Nh) {
    typedef typename CT<real>::t cplx;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_ok;
    cplx *tw = reinterpret_cast<cplx *>(smem_raw);
    cplx *tile = tw + N;
    const int box = blockIdx.x / 3, f = blockIdx.x % 3, kz0 = blockIdx.y * W, jy = blockIdx.z;
    constexpr int K = GeoN<N>::K, Kx = GeoN<N>::Kx, Kz = GeoN<N>::Kz, Kzp = GeoN<N>::Kzp;
    const cplx *src = A + box * GeoN<N>::bA + f * GeoN<N>::sA + (long long)jy * Kzp;
    cplx *dst = Nh + box * GeoN<N>::bB + f * GeoN<N>::sS + (long long)jy * Kzp;
    if constexpr (BULK) rows_issue<cplx, W>(g, tile, src + kz0, (long long)Kx * Kzp, N, min(W, Kzp - kz0), &bar);
    load_twiddles<real>(tw, twg, N, g.chk());
    if constexpr (BULK) {
        if (!rows_wait(&bar, &s_ok, g.err)) return;
    } else {
        __syncthreads();
    }
    auto load = [&](int n, int c) -> cplx {
        const int kz = kz0 + c;
        if (kz >= Kz) return cmk<cplx>(0.0, 0.0);
        return BULK ? tile[n * W + c] : DNS_LD(g, src + (long long)n * Kx * Kzp + kz);
    };
    auto store = [&](int n, int c, cplx v) {
        const int kz = kz0 + c;
        const int ix = row_to_compact<N>(n, K);
        if (kz < Kz && ix >= 0) DNS_ST(g, dst + (long long)ix * Kx * Kzp + kz, v);
    };
    TileFFT<real, N, W, T, -1, MAXR>::run(tile, W, tw, load, store);
}

// P5b: pointwise over the stored modes: Leray projection (Eq. pressure,
// NSfinal), viscous term and the RK4 stage (or the bare RHS / transform).
// Update of one stored mode (ix, iy, kz) of box `box` from its nonlinear
// term n0..n2: optional forcing, Leray projection (Eq. pressure / NSfinal),
// viscous term and the RK4 (or IF-RK4) stage, then omega^ of the next stage
// input for the next P1.
template <typename real, typename acc, int N>
__device__ __forceinline__ void p5_mode_update(const UpdateArgs<real, acc> &args, int box, int ix, int iy, int kz,
                                               typename CT<real>::t n0, typename CT<real>::t n1,
                                               typename CT<real>::t n2) {
    typedef typename CT<real>::t cplx;
    typedef typename CT<acc>::t cacc;
    typedef GeoN<N> G;
    constexpr long long sS = G::sS;
    const long long m = box * G::bS + ((long long)ix * G::Kx + iy) * G::Kzp + kz;  // state element, component 0
    const real nu = (real)(args.nu_box ? DNS_LD(args, args.nu_box + box) : args.nu);
    if (args.Fext && args.stage != -2) {
        const cplx f0 = DNS_LD(args, args.Fext + m), f1 = DNS_LD(args, args.Fext + sS + m),
                   f2 = DNS_LD(args, args.Fext + 2 * sS + m);
        n0 = cadd(n0, f0);
        n1 = cadd(n1, f1);
        n2 = cadd(n2, f2);
    }
    if (args.stage == -2) {  // bare forward transform (physical input)
        DNS_ST(args, args.dU + m, cmk<cacc>(n0.x, n0.y));
        DNS_ST(args, args.dU + sS + m, cmk<cacc>(n1.x, n1.y));
        DNS_ST(args, args.dU + 2 * sS + m, cmk<cacc>(n2.x, n2.y));
        return;
    }
    // every load of the mode before any store (the output arrays may alias
    // nothing the compiler can prove, so loads after a store would wait)
    const bool ifrk = args.ifrk && args.stage >= 0;
    cplx v[3];          // stage input (viscous term of classical RK4)
    cacc s0[3], s1[3];  // step-start state and accumulator
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        v[c] = cmk<cplx>(0.0, 0.0);
        s0[c] = s1[c] = cmk<cacc>(0.0, 0.0);
        if (!ifrk) v[c] = DNS_LD(args, args.U + c * sS + m);
        if (args.stage >= 0 && args.stage < 3) s0[c] = DNS_LD(args, args.U0 + c * sS + m);
        if (args.stage > 0) s1[c] = DNS_LD(args, args.U1 + c * sS + m);
    }
    const real kx = (real)compact_to_k(ix, G::K), ky = (real)compact_to_k(iy, G::K), kzr = (real)kz;
    const real k2 = kx * kx + ky * ky + kzr * kzr;
    const real inv = k2 > 0 ? (real)1 / k2 : (real)0;
    const real dre = (kx * n0.x + ky * n1.x + kzr * n2.x) * inv;
    const real dim = (kx * n0.y + ky * n1.y + kzr * n2.y) * inv;
    cplx x0, x1, x2;
    if (ifrk) {
        // integrating factor: the stage value is the projected nonlinear term
        // alone; the viscous decay enters through E1 = exp(-nu k^2 dt/2),
        // E2 = exp(-nu k^2 dt), evaluated in the accumulator precision
        const acc L = (acc)nu * (acc)k2;
        const acc e1 = exp(-L * (acc)(0.5 * args.dt)), e2 = exp(-L * (acc)args.dt);
        x0 = rk_update_if<real, acc>(args, m, cmk<cplx>(n0.x - kx * dre, n0.y - kx * dim), s0[0], s1[0], e1, e2);
        x1 = rk_update_if<real, acc>(args, sS + m, cmk<cplx>(n1.x - ky * dre, n1.y - ky * dim), s0[1], s1[1], e1,
                                     e2);
        x2 = rk_update_if<real, acc>(args, 2 * sS + m, cmk<cplx>(n2.x - kzr * dre, n2.y - kzr * dim), s0[2], s1[2],
                                     e1, e2);
    } else {
        const real vk = nu * k2;
        x0 = rk_update<real, acc>(args, m, cmk<cplx>(n0.x - kx * dre - vk * v[0].x, n0.y - kx * dim - vk * v[0].y),
                                  s0[0], s1[0]);
        x1 = rk_update<real, acc>(args, sS + m,
                                  cmk<cplx>(n1.x - ky * dre - vk * v[1].x, n1.y - ky * dim - vk * v[1].y), s0[1], s1[1]);
        x2 = rk_update<real, acc>(args, 2 * sS + m,
                                  cmk<cplx>(n2.x - kzr * dre - vk * v[2].x, n2.y - kzr * dim - vk * v[2].y), s0[2],
                                  s1[2]);
    }
    if (args.stage >= 0 && args.Om) {  // curl of the next stage input for the next P1
        cplx ox, oy, oz;
        curl_mode<cplx, real>(kx, ky, kzr, x0, x1, x2, ox, oy, oz);
        DNS_ST(args, args.Om + m, ox);
        DNS_ST(args, args.Om + sS + m, oy);
        DNS_ST(args, args.Om + 2 * sS + m, oz);
    }
}

// Grid: (stored modes of one field / blockDim.x, boxes); one mode per thread
// (no grid-stride loop: every thread's loads are independent, which keeps
// enough bytes in flight), its indices by divisions by compile-time constants.
template <typename real, typename acc, int N>
__global__ void k_p5b_update(const typename CT<real>::t *__restrict__ Nh, UpdateArgs<real, acc> args) {
    typedef typename CT<real>::t cplx;
    typedef GeoN<N> G;
    const int mm = blockIdx.x * blockDim.x + threadIdx.x, box = blockIdx.y;
    if (mm >= G::sS) return;
    const int kz = mm % G::Kzp;
    if (kz >= G::Kz) return;
    const int r = mm / G::Kzp;
    const int iy = r % G::Kx, ix = r / G::Kx;
    const long long nm = box * G::bB + mm;  // N^ lives in B, state layout
    const cplx n0 = DNS_LD(args, Nh + nm), n1 = DNS_LD(args, Nh + G::sS + nm), n2 = DNS_LD(args, Nh + 2 * G::sS + nm);
    p5_mode_update<real, acc, N>(args, box, ix, iy, kz, n0, n1, n2);
}

// P5a and P5b in one pass: a block transforms all three fields of one
// (ky, kz tile) along x (tile columns f*W + c), keeps the result in shared
// memory, and updates the Kx x W stored modes of the tile from it, so the
// nonlinear term never goes to HBM.
template <typename real, typename acc, int N, int W, int T, int MAXR>
__global__ void __launch_bounds__(T) k_p5_fused(Geo g, const typename CT<real>::t *__restrict__ twg,
                                                const typename CT<real>::t *__restrict__ A,
                                                UpdateArgs<real, acc> args) {
    typedef typename CT<real>::t cplx;
    constexpr int WT = 3 * W;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx *tw = reinterpret_cast<cplx *>(smem_raw);
    cplx *tile = tw + N;
    load_twiddles<real>(tw, twg, N, g.chk());
    __syncthreads();
    const int box = blockIdx.x, kz0 = blockIdx.y * W, jy = blockIdx.z;
    constexpr int K = GeoN<N>::K, Kx = GeoN<N>::Kx, Kz = GeoN<N>::Kz, Kzp = GeoN<N>::Kzp;
    const cplx *src = A + box * GeoN<N>::bA + (long long)jy * Kzp + kz0;
    auto load = [&](int n, int c) -> cplx {
        const int f = c / W, cc = c % W;
        if (kz0 + cc >= Kz) return cmk<cplx>(0.0, 0.0);
        return DNS_LD(g, src + f * GeoN<N>::sA + (long long)n * Kx * Kzp + cc);
    };
    auto tstore = [&](int n, int c, cplx v) { tile[n * WT + c] = v; };
    TileFFT<real, N, WT, T, -1, MAXR>::run(tile, WT, tw, load, tstore);
    for (int e = threadIdx.x; e < Kx * W; e += T) {
        const int ix = e / W, cc = e % W, kz = kz0 + cc;
        if (kz >= Kz) continue;
        const int kx = compact_to_k(ix, K);
        const int n = kx >= 0 ? kx : kx + N;
        const cplx *row = tile + n * WT + cc;
        p5_mode_update<real, acc, N>(args, box, ix, jy, kz, row[0], row[W], row[2 * W]);
    }
}

// ------------------------------------------------------------------- layout conversion
// full [3][N][N][N/2+1] <-> compact state layout; modes outside the kept set
// are dropped on the way in and zero on the way out.  One block per row:
// grid (y, x, component), the threads along kz (contiguous on both sides),
// so no index is divided.

// Kept rows in, to one or two compact buffers (cmp2 may be nullptr).
template <typename Tin, typename Tout, typename Tout2>
__global__ void k_full_to_compact(Geo g, const Tin *__restrict__ full, Tout *__restrict__ cmp,
                                  Tout2 *__restrict__ cmp2) {
    const int N = g.N, Nh = N / 2 + 1, K = g.K, Kx = g.Kx, Kz = g.Kz, Kzp = g.Kzp;
    const int iy = blockIdx.x, ix = blockIdx.y, c = blockIdx.z;
    const int fx = ix <= K ? ix : ix - Kx + N, fy = iy <= K ? iy : iy - Kx + N;
    const Tin *src = full + (((long long)c * N + fx) * N + fy) * Nh;
    const long long o = c * g.sS + ((long long)ix * Kx + iy) * Kzp;
    for (int kz = threadIdx.x; kz < Kz; kz += blockDim.x) {
        const Tin v = DNS_LD(g, src + kz);
        Tout a;
        a.x = v.x;
        a.y = v.y;
        DNS_ST(g, cmp + o + kz, a);
        if (cmp2) {
            Tout2 b;
            b.x = v.x;
            b.y = v.y;
            DNS_ST(g, cmp2 + o + kz, b);
        }
    }
}

template <typename Tin, typename Tout>
__global__ void k_compact_to_full(Geo g, const Tin *__restrict__ cmp, Tout *__restrict__ full) {
    const int N = g.N, Nh = N / 2 + 1, K = g.K, Kx = g.Kx, Kzp = g.Kzp;
    const int fy = blockIdx.x, fx = blockIdx.y, c = blockIdx.z;
    const int ix = fx <= K ? fx : (fx >= N - K ? fx - N + Kx : -1);
    const int iy = fy <= K ? fy : (fy >= N - K ? fy - N + Kx : -1);
    Tout *dst = full + (((long long)c * N + fx) * N + fy) * Nh;
    const bool kept = ix >= 0 && iy >= 0;
    const Tin *src = cmp + c * g.sS + (kept ? ((long long)ix * Kx + iy) * Kzp : 0);
    for (int kz = threadIdx.x; kz < Nh; kz += blockDim.x) {
        Tout o;
        o.x = 0;
        o.y = 0;
        if (kept && kz <= K) {
            const Tin v = DNS_LD(g, src + kz);
            o.x = v.x;
            o.y = v.y;
        }
        DNS_ST(g, dst + kz, o);
    }
}

// ------------------------------------------------------------------- diagnostics
// Partial sums per block of sum w |uhat|^2 and sum w |k|^2 |uhat|^2 (w = 1 at
// kz = 0, 2 otherwise), then one block adds the partials in a fixed order.
template <typename acc>
__global__ void k_energy_partials(Geo g, const typename CT<acc>::t *__restrict__ U, double *partials) {
    const int K = g.K, Kx = g.Kx, Kz = g.Kz, Kzp = g.Kzp;
    const long long total = (long long)Kx * Kx * Kz;
    double se = 0.0, sd = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int kz = (int)(e % Kz);
        const long long r = e / Kz;
        const int iy = (int)(r % Kx), ix = (int)(r / Kx);
        const double kx = compact_to_k(ix, K), ky = compact_to_k(iy, K);
        const double k2 = kx * kx + ky * ky + (double)kz * kz;
        const long long m = ((long long)ix * Kx + iy) * Kzp + kz;
        double p = 0.0;
        for (int c = 0; c < 3; ++c) {
            const typename CT<acc>::t v = DNS_LD(g, U + c * g.sS + m);
            p += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
        }
        const double w = kz == 0 ? 1.0 : 2.0;
        se += w * p;
        sd += w * k2 * p;
    }
    __shared__ double rs[2][1024 / 32];
    for (int o = 16; o > 0; o >>= 1) {
        se += __shfl_down_sync(0xffffffffu, se, o);
        sd += __shfl_down_sync(0xffffffffu, sd, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        rs[0][wid] = se;
        rs[1][wid] = sd;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += rs[0][w];
            b += rs[1][w];
        }
        DNS_ST(g, partials + 2 * blockIdx.x, a);
        DNS_ST(g, partials + 2 * blockIdx.x + 1, b);
    }
}

static __global__ void k_sum_partials(const double *partials, int nblocks, int stride, double *out) {
    // one thread per output column, fixed order
    const int c = threadIdx.x;
    if (c < stride) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += partials[b * stride + c];
        out[c] = s;
    }
}

// Shell spectrum: block s sums every mode with floor(|k| + 1/2) = s, i.e.
// (2s-1)^2 <= 4|k|^2 < (2s+1)^2, walking the kz run of each (kx, ky) column.
template <typename acc>
__global__ void k_spectrum(Geo g, const typename CT<acc>::t *__restrict__ U, double *Ek) {
    const int s = blockIdx.x;
    const int K = g.K, Kx = g.Kx, Kz = g.Kz, Kzp = g.Kzp;
    const long long lo4 = s == 0 ? 0 : (long long)(2 * s - 1) * (2 * s - 1);
    const long long hi4 = (long long)(2 * s + 1) * (2 * s + 1);
    double acc_s = 0.0;
    for (int col = threadIdx.x; col < Kx * Kx; col += blockDim.x) {
        const int ix = col / Kx, iy = col % Kx;
        const long long kx = compact_to_k(ix, K), ky = compact_to_k(iy, K);
        const long long r4 = 4 * (kx * kx + ky * ky);
        if (r4 >= hi4) continue;
        // smallest kz with r4 + 4 kz^2 >= lo4, and the first with >= hi4
        int a = 0;
        if (r4 < lo4) {
            a = (int)floor(sqrt((double)(lo4 - r4) / 4.0));
            while (a > 0 && r4 + 4LL * (a - 1) * (a - 1) >= lo4) --a;
            while (r4 + 4LL * a * a < lo4) ++a;
        }
        int b = (int)floor(sqrt((double)(hi4 - r4) / 4.0));
        while (b > 0 && r4 + 4LL * (b - 1) * (b - 1) >= hi4) --b;
        while (r4 + 4LL * b * b < hi4) ++b;
        if (b > Kz) b = Kz;
        const long long m0 = ((long long)ix * Kx + iy) * Kzp;
        for (int kz = a; kz < b; ++kz) {
            double p = 0.0;
            for (int c = 0; c < 3; ++c) {
                const typename CT<acc>::t v = DNS_LD(g, U + c * g.sS + m0 + kz);
                p += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
            }
            acc_s += (kz == 0 ? 1.0 : 2.0) * p;
        }
    }
    __shared__ double rs[1024 / 32];
    for (int o = 16; o > 0; o >>= 1) acc_s += __shfl_down_sync(0xffffffffu, acc_s, o);
    if ((threadIdx.x & 31) == 0) rs[threadIdx.x >> 5] = acc_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += rs[w];
        const double N3 = (double)g.N * g.N * g.N;
        DNS_ST(g, Ek + s, t / (2.0 * N3 * N3));
    }
}

}  // namespace dns
