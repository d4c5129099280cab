// The five passes of one evaluation of Eq. NSfinal, fused with their
// pointwise work (Mortensen, Sec. 2):
//
//   P1  curl (omega^ = i k x uhat) + inverse transform along x, 6 fields
//   P2  inverse transform along y, 6 fields
//   P3  inverse real transform along z of 6 fields, u x omega pointwise,
//       forward real transform along z of 3 fields (physical values never
//       leave shared memory)
//   P4  forward transform along y, 3 fields
//   P5  forward transform along x, then Leray projection, viscous term and
//       the RK4 stage update (or the bare right-hand side)
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
//   B      [6][N][N][Kzp]      after P2 (x, y physical); P3 writes N^ into fields 0..2
#pragma once

#include "dns_fft.cuh"

namespace dns {

struct Geo {
    int N, K, Kx, Kz, Kzp;
    long long sS;  // elements per state field  = Kx*Kx*Kzp
    long long sA;  // elements per A field      = N*Kx*Kzp
    long long sB;  // elements per B field      = N*N*Kzp
};

// Arguments of P5.  stage in 0..3 performs that RK4 stage; stage = -1 writes
// the right-hand side to dU instead.
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
    double nu;
    double adt;      // a_s * dt
    double bdt;      // b_s * dt
    int stage;
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
                                                                       int N) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = twg[i];
}

// ------------------------------------------------------------------- P1
template <typename real, int N, int W, int T>
__global__ void __launch_bounds__(T) k_p1_curl_xinv(Geo g, const typename CT<real>::t *__restrict__ twg,
                                                    const typename CT<real>::t *__restrict__ U,
                                                    typename CT<real>::t *__restrict__ A, real scale) {
    typedef typename CT<real>::t cplx;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx *tw = reinterpret_cast<cplx *>(smem_raw);
    cplx *tile = tw + N;
    load_twiddles<real>(tw, twg, N);
    __syncthreads();
    const int kz0 = blockIdx.x * W, jy = blockIdx.y, f = blockIdx.z;
    const int K = g.K, Kx = g.Kx, Kz = g.Kz, Kzp = g.Kzp;
    const real ky = (real)compact_to_k(jy, K);
    const long long sS = g.sS;
    auto load = [&](int n, int c) -> cplx {
        const int kz = kz0 + c;
        const int ix = row_to_compact<N>(n, K);
        cplx z;
        z.x = 0;
        z.y = 0;
        if (kz >= Kz || ix < 0) return z;
        const long long m = ((long long)ix * Kx + jy) * Kzp + kz;
        const real kx = (real)compact_to_k(ix, K), kzr = (real)kz;
        cplx v;
        if (f < 3) {
            v = U[f * sS + m];
        } else {
            // omega^ = i k x uhat
            cplx a, b;
            real ka, kb;
            if (f == 3) { a = U[2 * sS + m]; ka = ky; b = U[sS + m]; kb = kzr; }      // i(ky w - kz v)
            else if (f == 4) { a = U[m]; ka = kzr; b = U[2 * sS + m]; kb = kx; }     // i(kz u - kx w)
            else { a = U[sS + m]; ka = kx; b = U[m]; kb = ky; }                      // i(kx v - ky u)
            const real re = ka * a.x - kb * b.x, im = ka * a.y - kb * b.y;
            v.x = -im;
            v.y = re;
        }
        v.x *= scale;
        v.y *= scale;
        return v;
    };
    auto store = [&](int n, int c, cplx v) {
        const int kz = kz0 + c;
        if (kz < Kz) A[f * g.sA + ((long long)n * Kx + jy) * Kzp + kz] = v;
    };
    TileFFT<real, N, W, T, +1>::run(tile, W, tw, load, store);
}

// ------------------------------------------------------------------- P2
template <typename real, int N, int W, int T>
__global__ void __launch_bounds__(T) k_p2_yinv(Geo g, const typename CT<real>::t *__restrict__ twg,
                                               const typename CT<real>::t *__restrict__ A,
                                               typename CT<real>::t *__restrict__ B) {
    typedef typename CT<real>::t cplx;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx *tw = reinterpret_cast<cplx *>(smem_raw);
    cplx *tile = tw + N;
    load_twiddles<real>(tw, twg, N);
    __syncthreads();
    const int kz0 = blockIdx.x * W, x = blockIdx.y, f = blockIdx.z;
    const int K = g.K, Kx = g.Kx, Kz = g.Kz, Kzp = g.Kzp;
    const cplx *src = A + f * g.sA + (long long)x * Kx * Kzp;
    cplx *dst = B + f * g.sB + (long long)x * N * Kzp;
    auto load = [&](int n, int c) -> cplx {
        const int kz = kz0 + c;
        const int iy = row_to_compact<N>(n, K);
        cplx z;
        z.x = 0;
        z.y = 0;
        if (kz >= Kz || iy < 0) return z;
        return src[(long long)iy * Kzp + kz];
    };
    auto store = [&](int n, int c, cplx v) {
        const int kz = kz0 + c;
        if (kz < Kz) dst[(long long)n * Kzp + kz] = v;
    };
    TileFFT<real, N, W, T, +1>::run(tile, W, tw, load, store);
}

// ------------------------------------------------------------------- P3
// L lines (consecutive y at one x) per block.  Pairs of real fields share
// one complex transform: line p holds X_{2p} + i X_{2p+1}, extended to the
// full length by Hermitian symmetry; after the inverse transform the real
// and imaginary parts are the two physical fields.
template <typename real, int N, int L, int T>
__global__ void __launch_bounds__(T) k_p3_z_cross(Geo g, const typename CT<real>::t *__restrict__ twg,
                                                  typename CT<real>::t *__restrict__ B) {
    typedef typename CT<real>::t cplx;
    constexpr int LD = 3 * L + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx *tw = reinterpret_cast<cplx *>(smem_raw);
    cplx *tile = tw + N;
    load_twiddles<real>(tw, twg, N);
    const int K = g.K, Kz = g.Kz, Kzp = g.Kzp;
    const long long line0 = (long long)blockIdx.x * L;  // = x*N + y0
    const long long sB = g.sB;
    // zero the rows no stored mode reaches
    for (int e = threadIdx.x; e < (N - 2 * K - 1) * 3 * L; e += T) {
        const int n = K + 1 + e / (3 * L), c = e % (3 * L);
        tile[n * LD + c] = cmk<cplx>(0.0, 0.0);
    }
    // load + pack, consecutive threads on consecutive kz
    for (int e = threadIdx.x; e < 3 * L * Kz; e += T) {
        const int kz = e % Kz, pc = e / Kz, p = pc / L, c = pc % L;
        const long long off = (line0 + c) * Kzp + kz;
        cplx a = B[(2 * p) * sB + off];
        cplx b = B[(2 * p + 1) * sB + off];
        if (kz == 0) {
            a.y = 0;
            b.y = 0;
        }
        // Z[kz] = a + i b,  Z[N - kz] = conj(a) + i conj(b)
        tile[kz * LD + p * L + c] = cmk<cplx>(a.x - b.y, a.y + b.x);
        if (kz > 0) tile[(N - kz) * LD + p * L + c] = cmk<cplx>(a.x + b.y, b.x - a.y);
    }
    __syncthreads();
    auto tload = [&](int n, int c) -> cplx { return tile[n * LD + c]; };
    auto tstore = [&](int n, int c, cplx v) { tile[n * LD + c] = v; };
    TileFFT<real, N, 3 * L, T, +1>::run(tile, LD, tw, tload, tstore);
    // u x omega, component order c0 = a1 b2 - a2 b1, c1 = a2 b0 - a0 b2, c2 = a0 b1 - a1 b0
    for (int e = threadIdx.x; e < N * L; e += T) {
        const int n = e / L, c = e % L;
        const cplx p0 = tile[n * LD + c], p1 = tile[n * LD + L + c], p2 = tile[n * LD + 2 * L + c];
        const real ux = p0.x, uy = p0.y, uz = p1.x, wx = p1.y, wy = p2.x, wz = p2.y;
        const real nx = uy * wz - uz * wy;
        const real ny = uz * wx - ux * wz;
        const real nz = ux * wy - uy * wx;
        tile[n * LD + c] = cmk<cplx>(nx, ny);
        tile[n * LD + L + c] = cmk<cplx>(nz, 0.0);
    }
    __syncthreads();
    TileFFT<real, N, 2 * L, T, -1>::run(tile, LD, tw, tload, tstore);
    // unpack the two real transforms of line 0 and store kz <= K
    for (int e = threadIdx.x; e < L * Kz; e += T) {
        const int kz = e % Kz, c = e / Kz;
        const cplx za = tile[kz * LD + c];
        const cplx zm = tile[((N - kz) % N) * LD + c];
        const cplx zb = tile[kz * LD + L + c];
        const long long off = (line0 + c) * Kzp + kz;
        // X = (Z[k] + conj Z[N-k]) / 2,  Y = (Z[k] - conj Z[N-k]) / (2i)
        B[off] = cmk<cplx>(0.5 * (za.x + zm.x), 0.5 * (za.y - zm.y));
        B[sB + off] = cmk<cplx>(0.5 * (za.y + zm.y), -0.5 * (za.x - zm.x));
        B[2 * sB + off] = zb;
    }
}

// ------------------------------------------------------------------- physical input
// Forward real transform along z of a physical field u[3][N][N][N] (entry of
// a velocity given in physical space): lines (ux + i uy) and (uz + 0i).
template <typename real, typename ioreal, int N, int L, int T>
__global__ void __launch_bounds__(T) k_zfwd_real(Geo g, const typename CT<real>::t *__restrict__ twg,
                                                 const ioreal *__restrict__ u,
                                                 typename CT<real>::t *__restrict__ B) {
    typedef typename CT<real>::t cplx;
    constexpr int LD = 2 * L + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx *tw = reinterpret_cast<cplx *>(smem_raw);
    cplx *tile = tw + N;
    load_twiddles<real>(tw, twg, N);
    const int Kz = g.Kz, Kzp = g.Kzp;
    const long long line0 = (long long)blockIdx.x * L;
    const long long N3 = (long long)N * N * N;
    const long long sB = g.sB;
    for (int e = threadIdx.x; e < 2 * L * N; e += T) {
        const int z = e % N, pc = e / N, p = pc / L, c = pc % L;
        const long long off = (line0 + c) * N + z;
        if (p == 0) tile[z * LD + c] = cmk<cplx>((double)u[off], (double)u[N3 + off]);
        else tile[z * LD + L + c] = cmk<cplx>((double)u[2 * N3 + off], 0.0);
    }
    __syncthreads();
    auto tload = [&](int n, int c) -> cplx { return tile[n * LD + c]; };
    auto tstore = [&](int n, int c, cplx v) { tile[n * LD + c] = v; };
    TileFFT<real, N, 2 * L, T, -1>::run(tile, LD, tw, tload, tstore);
    for (int e = threadIdx.x; e < L * Kz; e += T) {
        const int kz = e % Kz, c = e / Kz;
        const cplx za = tile[kz * LD + c];
        const cplx zm = tile[((N - kz) % N) * LD + c];
        const cplx zb = tile[kz * LD + L + c];
        const long long off = (line0 + c) * Kzp + kz;
        B[off] = cmk<cplx>(0.5 * (za.x + zm.x), 0.5 * (za.y - zm.y));
        B[sB + off] = cmk<cplx>(0.5 * (za.y + zm.y), -0.5 * (za.x - zm.x));
        B[2 * sB + off] = zb;
    }
}

// ------------------------------------------------------------------- P4
template <typename real, int N, int W, int T>
__global__ void __launch_bounds__(T) k_p4_yfwd(Geo g, const typename CT<real>::t *__restrict__ twg,
                                               const typename CT<real>::t *__restrict__ B,
                                               typename CT<real>::t *__restrict__ A) {
    typedef typename CT<real>::t cplx;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx *tw = reinterpret_cast<cplx *>(smem_raw);
    cplx *tile = tw + N;
    load_twiddles<real>(tw, twg, N);
    __syncthreads();
    const int kz0 = blockIdx.x * W, x = blockIdx.y, f = blockIdx.z;
    const int K = g.K, Kx = g.Kx, Kz = g.Kz, Kzp = g.Kzp;
    const cplx *src = B + f * g.sB + (long long)x * N * Kzp;
    cplx *dst = A + f * g.sA + (long long)x * Kx * Kzp;
    auto load = [&](int n, int c) -> cplx {
        const int kz = kz0 + c;
        if (kz >= Kz) return cmk<cplx>(0.0, 0.0);
        return src[(long long)n * Kzp + kz];
    };
    auto store = [&](int n, int c, cplx v) {
        const int kz = kz0 + c;
        const int iy = row_to_compact<N>(n, K);
        if (kz < Kz && iy >= 0) dst[(long long)iy * Kzp + kz] = v;
    };
    TileFFT<real, N, W, T, -1>::run(tile, W, tw, load, store);
}

// ------------------------------------------------------------------- P5
template <typename real, typename acc>
__device__ __forceinline__ void rk_update(const UpdateArgs<real, acc> &a, long long m, int comp,
                                          long long sS, typename CT<real>::t du) {
    typedef typename CT<real>::t cplx;
    typedef typename CT<acc>::t cacc;
    const long long e = comp * sS + m;
    if (a.stage < 0) {
        a.dU[e] = cmk<cacc>((acc)du.x, (acc)du.y);
        return;
    }
    const acc dx = (acc)du.x, dy = (acc)du.y;
    const acc adt = (acc)a.adt, bdt = (acc)a.bdt;
    cacc u0, u1;
    if (a.stage < 3) u0 = a.U0[e];
    if (a.stage == 0) u1 = u0;
    else u1 = a.U1[e];
    u1.x += adt * dx;
    u1.y += adt * dy;
    if (a.stage < 3) {
        a.U1[e] = u1;
        a.Uout[e] = cmk<cplx>((double)(u0.x + bdt * dx), (double)(u0.y + bdt * dy));
    } else {
        a.U0out[e] = u1;
        if (a.Uout) a.Uout[e] = cmk<cplx>((double)u1.x, (double)u1.y);
    }
}

template <typename real, typename acc, int N, int W, int T>
__global__ void __launch_bounds__(T) k_p5_xfwd_update(Geo g, const typename CT<real>::t *__restrict__ twg,
                                                      const typename CT<real>::t *__restrict__ A,
                                                      UpdateArgs<real, acc> args) {
    typedef typename CT<real>::t cplx;
    typedef typename CT<acc>::t cacc;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx *tw = reinterpret_cast<cplx *>(smem_raw);
    cplx *tile = tw + N;
    cplx *res = tile + N * W;  // [3][Kx][W]: kept rows of the three transformed fields
    load_twiddles<real>(tw, twg, N);
    __syncthreads();
    const int kz0 = blockIdx.x * W, jy = blockIdx.y;
    const int K = g.K, Kx = g.Kx, Kz = g.Kz, Kzp = g.Kzp;
    const long long sS = g.sS;
#pragma unroll 1
    for (int f = 0; f < 3; ++f) {
        const cplx *src = A + f * g.sA + (long long)jy * Kzp;
        cplx *rf = res + f * Kx * W;
        auto load = [&](int n, int c) -> cplx {
            const int kz = kz0 + c;
            if (kz >= Kz) return cmk<cplx>(0.0, 0.0);
            return src[(long long)n * Kx * Kzp + kz];
        };
        auto store = [&](int n, int c, cplx v) {
            const int ix = row_to_compact<N>(n, K);
            if (ix >= 0) rf[ix * W + c] = v;
        };
        TileFFT<real, N, W, T, -1>::run(tile, W, tw, load, store);
    }
    // pointwise: consecutive threads on consecutive kz
    const real ky = (real)compact_to_k(jy, K);
    const real nu = (real)args.nu;
    for (int e = threadIdx.x; e < Kx * W; e += T) {
        const int ix = e / W, c = e % W, kz = kz0 + c;
        if (kz >= Kz) continue;
        const cplx n0 = res[e], n1 = res[Kx * W + e], n2 = res[2 * Kx * W + e];
        const long long m = ((long long)ix * Kx + jy) * Kzp + kz;
        if (args.stage == -2) {  // bare forward transform (physical input)
            args.dU[m] = cmk<cacc>(n0.x, n0.y);
            args.dU[sS + m] = cmk<cacc>(n1.x, n1.y);
            args.dU[2 * sS + m] = cmk<cacc>(n2.x, n2.y);
            continue;
        }
        const real kx = (real)compact_to_k(ix, K), kzr = (real)kz;
        const real k2 = kx * kx + ky * ky + kzr * kzr;
        const real inv = k2 > 0 ? (real)1 / k2 : (real)0;
        // Leray projection: N^ - k (k . N^) / |k|^2  (Eq. pressure, NSfinal)
        const real dre = (kx * n0.x + ky * n1.x + kzr * n2.x) * inv;
        const real dim = (kx * n0.y + ky * n1.y + kzr * n2.y) * inv;
        const cplx u0 = args.U[m], u1 = args.U[sS + m], u2 = args.U[2 * sS + m];
        const real vk = nu * k2;
        rk_update<real, acc>(args, m, 0, sS, cmk<cplx>(n0.x - kx * dre - vk * u0.x, n0.y - kx * dim - vk * u0.y));
        rk_update<real, acc>(args, m, 1, sS, cmk<cplx>(n1.x - ky * dre - vk * u1.x, n1.y - ky * dim - vk * u1.y));
        rk_update<real, acc>(args, m, 2, sS, cmk<cplx>(n2.x - kzr * dre - vk * u2.x, n2.y - kzr * dim - vk * u2.y));
    }
}

// ------------------------------------------------------------------- layout conversion
// full [3][N][N][N/2+1] <-> compact state layout; modes outside the kept set
// are dropped on the way in and zero on the way out.
template <typename Tin, typename Tout>
__global__ void k_full_to_compact(Geo g, const Tin *__restrict__ full, Tout *__restrict__ cmp) {
    const int N = g.N, Nh = N / 2 + 1, K = g.K, Kx = g.Kx, Kz = g.Kz, Kzp = g.Kzp;
    const long long total = 3LL * Kx * Kx * Kz;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int kz = (int)(e % Kz);
        const long long r = e / Kz;
        const int iy = (int)(r % Kx), ix = (int)((r / Kx) % Kx), c = (int)(r / ((long long)Kx * Kx));
        const int fx = ix <= K ? ix : ix - Kx + N, fy = iy <= K ? iy : iy - Kx + N;
        const Tin v = full[(((long long)c * N + fx) * N + fy) * Nh + kz];
        Tout o;
        o.x = v.x;
        o.y = v.y;
        cmp[c * g.sS + ((long long)ix * Kx + iy) * Kzp + kz] = o;
    }
}

template <typename Tin, typename Tout>
__global__ void k_compact_to_full(Geo g, const Tin *__restrict__ cmp, Tout *__restrict__ full) {
    const int N = g.N, Nh = N / 2 + 1, K = g.K, Kx = g.Kx, Kzp = g.Kzp;
    const long long total = 3LL * N * N * Nh;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int kz = (int)(e % Nh);
        const long long r = e / Nh;
        const int fy = (int)(r % N), fx = (int)((r / N) % N), c = (int)(r / ((long long)N * N));
        const int ix = fx <= K ? fx : (fx >= N - K ? fx - N + Kx : -1);
        const int iy = fy <= K ? fy : (fy >= N - K ? fy - N + Kx : -1);
        Tout o;
        o.x = 0;
        o.y = 0;
        if (ix >= 0 && iy >= 0 && kz <= K) {
            const Tin v = cmp[c * g.sS + ((long long)ix * Kx + iy) * Kzp + kz];
            o.x = v.x;
            o.y = v.y;
        }
        full[e] = o;
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
            const typename CT<acc>::t v = U[c * g.sS + m];
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
        partials[2 * blockIdx.x] = a;
        partials[2 * blockIdx.x + 1] = b;
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
                const typename CT<acc>::t v = U[c * g.sS + m0 + kz];
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
        Ek[s] = t / (2.0 * N3 * N3);
    }
}

}  // namespace dns
