// Tile FFT engine for the pseudo-spectral solver (sm_103a).
//
// A "tile" is a block of W independent lines of length N held in shared
// memory as tile[n * ld + c] (row n = position along the transformed axis,
// column c = line).  One thread block transforms all W lines together with a
// self-sorting (Stockham) mixed-radix schedule: for a stage of radix R that
// follows stages whose radices multiply to Ns, butterfly j (0 <= j < N/R)
// of every line reads x[j + r N/R], multiplies input r by w_{Ns R}^{r (j mod
// Ns)}, takes an R-point DFT and writes output r to
// (j / Ns) Ns R + (j mod Ns) + r Ns.  After the last stage the line is in
// natural order (Eq. ffteq: X[k] = sum_n x[n] exp(sign 2 pi i k n / N)).
//
// Consecutive threads take consecutive columns, so with 128-byte rows every
// warp access to the tile is free of bank conflicts, and the first stage
// (read through a Load functor, usually straight from HBM) and the last
// stage (written through a Store functor) are coalesced along the columns.
// Each stage keeps all of a thread's butterflies in registers between a read
// phase and a write phase separated by __syncthreads(), so one buffer serves
// in place.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dns_check.cuh"

namespace dns {

template <typename R> struct CT;
template <> struct CT<float> { typedef float2 t; };
template <> struct CT<double> { typedef double2 t; };
template <typename C> struct RealOf;
template <> struct RealOf<float2> { typedef float t; };
template <> struct RealOf<double2> { typedef double t; };

template <typename T> __device__ __forceinline__ T cmk(double x, double y) {
    T r;
    r.x = (decltype(r.x))x;
    r.y = (decltype(r.y))y;
    return r;
}
template <typename T> __device__ __forceinline__ T cadd(T a, T b) { T r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename T> __device__ __forceinline__ T csub(T a, T b) { T r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename T> __device__ __forceinline__ T cmul(T a, T b) {
    T r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
template <typename T> __device__ __forceinline__ T cconj(T a) { a.y = -a.y; return a; }
// multiply by sign * i
template <int SIGN, typename T> __device__ __forceinline__ T cmul_si(T a) {
    T r;
    if (SIGN > 0) { r.x = -a.y; r.y = a.x; }
    else { r.x = a.y; r.y = -a.x; }
    return r;
}
template <typename T, typename S> __device__ __forceinline__ T cscale(T a, S s) { a.x *= s; a.y *= s; return a; }

// ---------------------------------------------------------------------------
// Radix plan: N = 3^b * 2^a.  b radix-3 stages first, then the power of two
// split into the fewest stages whose radices are at most MAXR (8, 16 or
// 32), as equal as possible, smaller first: 2^9 with MAXR 8 -> 8*8*8, with
// 32 -> 16*32; 2^10 with 8 -> 4*4*8*8; 9 * 2^5 with 8 -> 3*3*4*8.
struct FftPlan {
    int nst;
    int r[8];
    int ns[8];  // product of the radices of the earlier stages
};

__host__ __device__ constexpr FftPlan make_plan(int N, int MAXR = 8) {
    FftPlan p{0, {0, 0, 0, 0, 0, 0, 0, 0}, {0, 0, 0, 0, 0, 0, 0, 0}};
    int n = N;
    while (n % 3 == 0) { p.r[p.nst++] = 3; n /= 3; }
    int a = 0;
    while ((1 << a) < n) ++a;
    int lmax = MAXR >= 32 ? 5 : (MAXR >= 16 ? 4 : 3);
    int ns_ = (a + lmax - 1) / lmax;  // number of power-of-two stages
    for (int s = 0; s < ns_; ++s) {  // smaller radices first
        int e = a / ns_ + (s >= ns_ - a % ns_ ? 1 : 0);
        p.r[p.nst++] = 1 << e;
    }
    int ns = 1;
    for (int s = 0; s < p.nst; ++s) { p.ns[s] = ns; ns *= p.r[s]; }
    return p;
}

// The same radices in the opposite order (larger first): an inverse run
// with this plan ends with the radix a forward run with make_plan starts
// with, so its last stage leaves each work item exactly the points the
// forward first stage needs (positions j + r N / R).
__host__ __device__ constexpr FftPlan make_plan_rev(int N, int MAXR = 8) {
    FftPlan f = make_plan(N, MAXR);
    FftPlan p{f.nst, {0, 0, 0, 0, 0, 0, 0, 0}, {0, 0, 0, 0, 0, 0, 0, 0}};
    for (int s = 0; s < f.nst; ++s) p.r[s] = f.r[f.nst - 1 - s];
    int ns = 1;
    for (int s = 0; s < p.nst; ++s) { p.ns[s] = ns; ns *= p.r[s]; }
    return p;
}

__host__ __device__ constexpr FftPlan plan_of(int N, int MAXR, bool rev) {
    return rev ? make_plan_rev(N, MAXR) : make_plan(N, MAXR);
}

__host__ __device__ constexpr int plan_max_radix(int N, int MAXR = 8) {
    FftPlan p = make_plan(N, MAXR);
    int m = 1;
    for (int s = 0; s < p.nst; ++s) m = p.r[s] > m ? p.r[s] : m;
    return m;
}

// cos(2 pi m / 32), m = 0..8 (first quadrant; the rest follow by symmetry)
__host__ __device__ constexpr double kCos32(int m) {
    return m == 0 ? 1.0
         : m == 1 ? 0.980785280403230449126
         : m == 2 ? 0.923879532511286756128
         : m == 3 ? 0.831469612302545237079
         : m == 4 ? 0.707106781186547524401
         : m == 5 ? 0.555570233019602224743
         : m == 6 ? 0.382683432365089771728
         : m == 7 ? 0.195090322016128267848
         : 0.0;
}
// exp(2 pi i m / 32) as (cos, sin), any m >= 0
__host__ __device__ constexpr double w32_re(int m) {
    return (m % 32) / 8 == 0 ? kCos32(m % 8)
         : (m % 32) / 8 == 1 ? -kCos32(8 - m % 8)
         : (m % 32) / 8 == 2 ? -kCos32(m % 8)
         : kCos32(8 - m % 8);
}
__host__ __device__ constexpr double w32_im(int m) {
    return (m % 32) / 8 == 0 ? kCos32(8 - m % 8)
         : (m % 32) / 8 == 1 ? kCos32(m % 8)
         : (m % 32) / 8 == 2 ? -kCos32(8 - m % 8)
         : -kCos32(m % 8);
}

// ---------------------------------------------------------------------------
// Small DFTs in registers: X[k] = sum_n v[n] exp(SIGN 2 pi i k n / R).
template <int P, int Q, int SIGN, typename T> __device__ __forceinline__ void dft_pq(T *v);

template <int R, int SIGN, typename T> __device__ __forceinline__ void dft(T *v) {
    typedef typename RealOf<T>::t real;
    if constexpr (R == 2) {
        T a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (R == 3) {
        const real h = (real)0.86602540378443864676;  // sqrt(3)/2
        T t1 = cadd(v[1], v[2]);
        T t2 = csub(v[0], cscale(t1, (real)0.5));
        T t3 = cscale(csub(v[1], v[2]), (real)SIGN * h);
        v[0] = cadd(v[0], t1);
        v[1] = cmk<T>(t2.x - t3.y, t2.y + t3.x);
        v[2] = cmk<T>(t2.x + t3.y, t2.y - t3.x);
    } else if constexpr (R == 4) {
        T s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
        T s13 = cadd(v[1], v[3]), d13 = cmul_si<SIGN>(csub(v[1], v[3]));
        v[0] = cadd(s02, s13);
        v[2] = csub(s02, s13);
        v[1] = cadd(d02, d13);
        v[3] = csub(d02, d13);
    } else if constexpr (R == 8) {
        T e[4] = {v[0], v[2], v[4], v[6]};
        T o[4] = {v[1], v[3], v[5], v[7]};
        dft<4, SIGN>(e);
        dft<4, SIGN>(o);
        const real c = (real)0.70710678118654752440;  // 1/sqrt(2)
        // w^1 = (1 + SIGN i)/sqrt2, w^2 = SIGN i, w^3 = (-1 + SIGN i)/sqrt2
        T o1 = cmk<T>((o[1].x - SIGN * o[1].y) * c, (o[1].y + SIGN * o[1].x) * c);
        T o2 = cmul_si<SIGN>(o[2]);
        T o3 = cmk<T>((-o[3].x - SIGN * o[3].y) * c, (SIGN * o[3].x - o[3].y) * c);
        v[0] = cadd(e[0], o[0]);
        v[4] = csub(e[0], o[0]);
        v[1] = cadd(e[1], o1);
        v[5] = csub(e[1], o1);
        v[2] = cadd(e[2], o2);
        v[6] = csub(e[2], o2);
        v[3] = cadd(e[3], o3);
        v[7] = csub(e[3], o3);
    } else if constexpr (R == 16) {
        dft_pq<4, 4, SIGN>(v);
    } else if constexpr (R == 32) {
        dft_pq<8, 4, SIGN>(v);
    } else {
        static_assert(R == 2 || R == 3 || R == 4 || R == 8 || R == 16 || R == 32, "unsupported radix");
    }
}

// Composite DFT of length P*Q in registers (Cooley-Tukey with n = Q n1 + n2,
// k = k1 + P k2): P-point DFTs over n1, twiddles w_{PQ}^{n2 k1}, Q-point DFTs
// over n2.  P*Q divides 32, so the twiddles are compile-time constants.
template <int P, int Q, int SIGN, typename T> __device__ __forceinline__ void dft_pq(T *v) {
    typedef typename RealOf<T>::t real;
    constexpr int PQ = P * Q;
    T y[Q][P];
#pragma unroll
    for (int n2 = 0; n2 < Q; ++n2) {
        T t[P];
#pragma unroll
        for (int n1 = 0; n1 < P; ++n1) t[n1] = v[Q * n1 + n2];
        dft<P, SIGN>(t);
#pragma unroll
        for (int k1 = 0; k1 < P; ++k1) y[n2][k1] = t[k1];
    }
#pragma unroll
    for (int n2 = 1; n2 < Q; ++n2) {
#pragma unroll
        for (int k1 = 1; k1 < P; ++k1) {
            const int m = ((n2 * k1) % PQ) * (32 / PQ);
            if (m == 8) {
                y[n2][k1] = cmul_si<SIGN>(y[n2][k1]);
            } else if (m == 24) {
                y[n2][k1] = cmul_si<-SIGN>(y[n2][k1]);
            } else if (m == 16) {
                y[n2][k1] = cscale(y[n2][k1], (real)-1);
            } else if (m != 0) {
                T w;
                w.x = (real)w32_re(m);
                w.y = (real)(SIGN * w32_im(m));
                y[n2][k1] = cmul(y[n2][k1], w);
            }
        }
    }
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) {
        T t[Q];
#pragma unroll
        for (int n2 = 0; n2 < Q; ++n2) t[n2] = y[n2][k1];
        dft<Q, SIGN>(t);
#pragma unroll
        for (int k2 = 0; k2 < Q; ++k2) v[k1 + P * k2] = t[k2];
    }
}

// ---------------------------------------------------------------------------
// The engine.  tw[m] = exp(-2 pi i m / N) (forward table); SIGN = +1 uses
// its conjugate.  Load(n, c) -> value of row n of line c for the first
// stage; Store(n, c, v) consumes row n of line c after the last stage.
template <typename real, int N, int W, int T, int SIGN, int MAXR = 8, int S = 0>
struct TileFFT {
    typedef typename CT<real>::t cplx;
    template <class Load, class Store>
    static __device__ __forceinline__ void run(cplx *tile, int ld, const cplx *tw, const Load &load,
                                               const Store &store) {
        constexpr FftPlan P = make_plan(N, MAXR);
        constexpr int R = P.r[S];
        constexpr int Ns = P.ns[S];
        constexpr int NB = N / R;
        constexpr int TOT = NB * W;
        constexpr int Q = (TOT + T - 1) / T;
        constexpr bool first = (S == 0);
        constexpr bool last = (S == P.nst - 1);
        constexpr int TWS = N / (Ns * R);
        cplx v[Q][R];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int idx = (int)threadIdx.x + q * T;
            if (Q * T == TOT || idx < TOT) {
                const int c = idx % W, j = idx / W;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int n = j + r * NB;
                    if constexpr (first) v[q][r] = load(n, c);
                    else v[q][r] = tile[n * ld + c];
                }
                if constexpr (!first) {
                    const int k = j % Ns;
#pragma unroll
                    for (int r = 1; r < R; ++r) {
                        cplx w = tw[r * k * TWS];
                        if (SIGN > 0) w.y = -w.y;
                        v[q][r] = cmul(v[q][r], w);
                    }
                }
                dft<R, SIGN>(v[q]);
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int idx = (int)threadIdx.x + q * T;
            if (Q * T == TOT || idx < TOT) {
                const int c = idx % W, j = idx / W;
                const int base = (j / Ns) * Ns * R + (j % Ns);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int n = base + r * Ns;
                    if constexpr (last) store(n, c, v[q][r]);
                    else tile[n * ld + c] = v[q][r];
                }
            }
        }
        __syncthreads();
        if constexpr (!last) TileFFT<real, N, W, T, SIGN, MAXR, S + 1>::run(tile, ld, tw, load, store);
    }
};

// ---------------------------------------------------------------------------
// Row-mapped variant for lines that are contiguous in memory: NV lines of
// length N in shared memory as tile[v * ldr + n + n/16] (one pad element per
// 16 keeps every stage's accesses free of bank conflicts, including the
// stride-R writes of a first stage).  Work item (v, j) = butterfly j of line
// v, consecutive threads on consecutive j, so a first stage reading straight
// from HBM is coalesced along the line.
__host__ __device__ constexpr int row_ld(int N) { return N + N / 16; }
__device__ __forceinline__ int radd(int n) { return n + (n >> 4); }

// Per-stage twiddle tables for the row engine.  In stage s >= 1 work item j
// multiplies input r by w^(r k TWS), k = j mod Ns; neighbouring items read
// entries r k TWS apart in the N-entry table, which puts many lanes of a warp
// on one shared-memory bank for the larger r.  The table of stage s instead
// holds, per k, the factors of a split r = R1 a + b: w^(b k TWS) for
// b = 1..R1-1 and w^(R1 a k TWS) for a = 1..R/R1-1 (radix 32: 8 x 4, 16:
// 4 x 4, smaller radices unsplit), each factor one product away; rows are
// padded to an odd length, so a warp's lanes read an odd stride apart (free
// of bank conflicts) and a radix-32 item reads 10 entries instead of 31.
// The tables of all stages follow each other; twt_size rounds their total
// up to even so what follows stays 16-byte aligned.
__host__ __device__ constexpr int twt_r1(int R) { return R == 32 ? 8 : (R == 16 ? 4 : R); }
__host__ __device__ constexpr int twt_row(int R) {
    const int e = (twt_r1(R) - 1) + (R / twt_r1(R) - 1);
    return e % 2 ? e : e + 1;
}
__host__ __device__ constexpr int twt_offset(int N, int MAXR, int S, bool rev = false) {
    FftPlan p = plan_of(N, MAXR, rev);
    int off = 0;
    for (int s = 1; s < S && s < p.nst; ++s) off += p.ns[s] * twt_row(p.r[s]);
    return off;
}
__host__ __device__ constexpr int twt_size(int N, int MAXR, bool rev = false) {
    const int t = twt_offset(N, MAXR, 64, rev);
    return (t + 1) / 2 * 2;
}
// Fill the stage tables of one plan (twt_size entries at twt) from the
// N-entry table in global memory; every thread of the block takes part.
// Kernels that also run the reversed plan keep its tables right after the
// forward plan's: tw [N] | forward tables | reversed tables.
template <typename cplx, int N, int MAXR, bool REV = false, int S = 1>
__device__ __forceinline__ void build_twt(cplx *twt, const cplx *twg, const Chk &ck = Chk{}) {
    constexpr FftPlan P = plan_of(N, MAXR, REV);
    if constexpr (S < P.nst) {
        constexpr int R = P.r[S], Ns = P.ns[S], TWS = N / (Ns * R), off = twt_offset(N, MAXR, S, REV);
        constexpr int R1 = twt_r1(R), ROW = twt_row(R);
        for (int e = threadIdx.x; e < Ns * ROW; e += blockDim.x) {
            const int k = e / ROW, i = e % ROW;
            int r = 0;  // padding entries repeat w^0
            if (i < R1 - 1) r = i + 1;
            else if (i < R1 - 1 + R / R1 - 1) r = R1 * (i - (R1 - 1) + 1);
            twt[off + e] = DNS_LD(ck, twg + r * k * TWS);
        }
        build_twt<cplx, N, MAXR, REV, S + 1>(twt, twg, ck);
    }
}
// The R - 1 twiddles w^(r k TWS), r = 1..R-1, of one work item from its row
// tk of a stage table (w[0] is left unset).
template <int R, typename cplx> __device__ __forceinline__ void stage_twiddles(const cplx *tk, cplx (&w)[R]) {
    constexpr int R1 = twt_r1(R), R2 = R / R1;
    cplx wb[R1], wa[R2];
#pragma unroll
    for (int b = 1; b < R1; ++b) wb[b] = tk[b - 1];
#pragma unroll
    for (int a = 1; a < R2; ++a) wa[a] = tk[R1 - 1 + a - 1];
#pragma unroll
    for (int r = 1; r < R; ++r) {
        const int a = r / R1, b = r % R1;
        w[r] = a == 0 ? wb[b] : (b == 0 ? wa[a] : cmul(wa[a], wb[b]));
    }
}

// ONE = true runs stage S alone (its output stays in the tile unless S is
// the last stage), so a caller can act between the first stage and the rest.
// TWT = true reads the twiddles of stages >= 1 from the per-stage tables at
// tw + N (see build_twt) instead of the N-entry table.  REVP runs the
// reversed plan (make_plan_rev); SKIPLAST stops before the plan's last
// stage, leaving its input in the tile.
template <typename real, int N, int NV, int T, int SIGN, int MAXR, int S = 0, bool ONE = false, bool TWT = false,
          bool REVP = false, bool SKIPLAST = false>
struct RowFFT {
    typedef typename CT<real>::t cplx;
    // Load(v, n): first-stage input; Store(v, n, x): last-stage output.
    template <class Load, class Store>
    static __device__ __forceinline__ void run(cplx *tile, const cplx *tw, const Load &load, const Store &store) {
        constexpr FftPlan P = plan_of(N, MAXR, REVP);
        constexpr int R = P.r[S];
        constexpr int Ns = P.ns[S];
        constexpr int NB = N / R;
        constexpr int TOT = NB * NV;
        constexpr int Q = (TOT + T - 1) / T;
        constexpr bool first = (S == 0);
        constexpr bool last = (S == P.nst - 1);
        constexpr int TWS = N / (Ns * R);
        constexpr int LDR = row_ld(N);
        cplx v[Q][R];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int idx = (int)threadIdx.x + q * T;
            if (Q * T == TOT || idx < TOT) {
                const int vl = idx / NB, j = idx % NB;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int n = j + r * NB;
                    if constexpr (first) v[q][r] = load(vl, n);
                    else v[q][r] = tile[vl * LDR + radd(n)];
                }
                if constexpr (!first) {
                    const int k = j % Ns;
                    cplx w[R];
                    if constexpr (TWT) {
                        stage_twiddles<R>(tw + N + (REVP ? twt_size(N, MAXR) : 0) + twt_offset(N, MAXR, S, REVP) +
                                              k * twt_row(R),
                                          w);
                    } else {
#pragma unroll
                        for (int r = 1; r < R; ++r) w[r] = tw[r * k * TWS];
                    }
#pragma unroll
                    for (int r = 1; r < R; ++r) {
                        if (SIGN > 0) w[r].y = -w[r].y;
                        v[q][r] = cmul(v[q][r], w[r]);
                    }
                }
                dft<R, SIGN>(v[q]);
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int idx = (int)threadIdx.x + q * T;
            if (Q * T == TOT || idx < TOT) {
                const int vl = idx / NB, j = idx % NB;
                const int base = (j / Ns) * Ns * R + (j % Ns);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int n = base + r * Ns;
                    if constexpr (last) store(vl, n, v[q][r]);
                    else tile[vl * LDR + radd(n)] = v[q][r];
                }
            }
        }
        __syncthreads();
        if constexpr (!last && !ONE && !(SKIPLAST && S + 2 == P.nst))
            RowFFT<real, N, NV, T, SIGN, MAXR, S + 1, false, TWT, REVP, SKIPLAST>::run(tile, tw, load, store);
    }
};

// Threads for a W-column tile so that no thread holds more than BUDGET
// complex values in registers in any stage (BUDGET >= the largest radix).
__host__ __device__ constexpr int tile_threads(int N, int W, int BUDGET) {
    int t = (N * W + BUDGET - 1) / BUDGET;
    t = ((t + 31) / 32) * 32;
    return t < 32 ? 32 : (t > 1024 ? 1024 : t);
}

}  // namespace dns
