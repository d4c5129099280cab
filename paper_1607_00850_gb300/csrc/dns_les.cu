// Learned subgrid closure for a coarse LES (not in the paper): training data
// from the DNS, a 3-layer periodic 3x3x3 convolutional network (9 filtered
// velocity gradients -> 32 -> 32 -> 6 subgrid stresses, GELU, BF16 operands,
// FP32 accumulation) trained with Adam, and the closure term in the LES
// right-hand side.  C ABI in include/dns.h (dns_net_*, dns_les_*).
//
// Convolutions are implicit GEMMs on the tensor cores with mma.sync
// m16n8k16 (BF16 in, FP32 accumulate): M = voxels, N = output channels,
// K = 27 taps x input channels.  Activations are voxel-major [V][C] BF16 so a
// tap's K slice is contiguous; weights are [Cout][27][Cin] BF16.  The input
// gradient is the same convolution with flipped taps and transposed weights;
// the weight gradient is a per-tap GEMM over voxel chunks (dY^T X_t) with
// both operands transposed through shared memory, reduced over chunks in a
// fixed order.
#include "dns.h"
#include "dns_internal.h"
#include "dns_les.cuh"
#include "dns_tc.cuh"

#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

namespace {
// A named NVTX range for the duration of an entry point: a timeline tool
// (Nsight Systems or ncu's NVTX filters) shows each C-ABI call; with no tool
// attached the push and pop do nothing.
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};
}  // namespace

namespace dns {
namespace les {

// ---------------------------------------------------------------- complex FFT launchers
template <int N> struct C2C {
    static constexpr int W = 16;
    static constexpr int T = N * W / 16 < 32 ? 32 : (N * W / 16 > 1024 ? 1024 : N * W / 16);
    static constexpr int L = 16;  // z lines per block
    static constexpr int TZ = N * L / 16 < 32 ? 32 : (N * L / 16 > 1024 ? 1024 : N * L / 16);
    static constexpr size_t smem_col = sizeof(float2) * (N + N * W);
    static constexpr size_t smem_row = sizeof(float2) * (N + L * row_ld(N));
    template <int SIGN> static cudaError_t run(float2 *a, const float2 *tw, int nfield, cudaStream_t st) {
        static_assert(N % L == 0 || N < L, "lines");
        cudaError_t e;
        auto kx = k_c2c_axis<N, W, T, SIGN, 0>;
        auto ky = k_c2c_axis<N, W, T, SIGN, 1>;
        auto kz = k_c2c_axis<N, L, TZ, SIGN, 2>;
        if ((e = cudaFuncSetAttribute(kx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_col)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(ky, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_col)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(kz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_row)) != cudaSuccess) return e;
        const dim3 gc(N / W, N, nfield);
        kx<<<gc, T, smem_col, st>>>(a, tw);
        ky<<<gc, T, smem_col, st>>>(a, tw);
        kz<<<(unsigned)((long long)N * N * nfield / L), TZ, smem_row, st>>>(a, tw);
        return cudaGetLastError();
    }
};

static cudaError_t c2c(int N, float2 *a, const float2 *tw, int nfield, int sign, cudaStream_t st) {
    switch (N) {
#define DNS_C2C(n) \
    case n: return sign < 0 ? C2C<n>::run<-1>(a, tw, nfield, st) : C2C<n>::run<+1>(a, tw, nfield, st);
        DNS_C2C(16) DNS_C2C(32) DNS_C2C(64) DNS_C2C(128) DNS_C2C(256)
#undef DNS_C2C
        default: return cudaErrorInvalidValue;
    }
}

static bool c2c_supported(int N) { return N == 16 || N == 32 || N == 64 || N == 128 || N == 256; }

static inline unsigned nblk(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

constexpr size_t kMaxSmemLes = 226 * 1024;  // dynamic shared memory a block may use (+ its static barriers)

// ---------------------------------------------------------------- network kernels
__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float x) {
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

__device__ __forceinline__ uint32_t ld_b32(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

__device__ __forceinline__ void mma_bf16(float *d, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ long long nbr(int n, int x, int y, int z, int t) {
    const int dx = t / 9 - 1, dy = (t / 3) % 3 - 1, dz = t % 3 - 1;
    x = (x + dx + n) % n;
    y = (y + dy + n) % n;
    z = (z + dz + n) % n;
    return ((long long)x * n + y) * n + z;
}

enum { EPI_HIDDEN = 0, EPI_OUT = 1, EPI_DGRAD = 2 };

// Y[v][o] = b[o] + sum_{t,c} X[v + off(t)][c] W[o][t][c].  A block of 4
// warps stages the layer's weights in shared memory once (rows padded by 8
// BF16 so the B-fragment reads of a warp hit 32 distinct banks); each warp
// computes MT m-tiles of 16 voxels along z (an m-tile never crosses a z
// line: n % 16 == 0) for all COUT outputs, so one B fragment feeds MT MMAs
// and one A fragment NT MMAs.  Epilogues:
//   EPI_HIDDEN: Z = Y (float) and A = bf16(gelu(Z));  EPI_OUT: Z = Y;
//   EPI_DGRAD:  A = bf16(Y * gelu'(Zp)) (Y is dL/da of the layer below).
constexpr int CONV_MT = 4;
constexpr int CONV_VOX = 4 * CONV_MT * 16;  // voxels per block

template <int CIN> __host__ __device__ constexpr int conv_ldw() { return 27 * CIN + 8; }
template <int CIN, int COUT> constexpr size_t conv_smem() { return sizeof(__nv_bfloat16) * COUT * conv_ldw<CIN>(); }

template <int CIN, int COUT, int EPI>
__global__ void __launch_bounds__(128) k_conv(int n, const __nv_bfloat16 *__restrict__ X,
                                              const __nv_bfloat16 *__restrict__ W, const float *__restrict__ bias,
                                              float *__restrict__ Z, __nv_bfloat16 *__restrict__ A,
                                              const float *__restrict__ Zp) {
    constexpr int NT = COUT / 8, MT = CONV_MT, LDW = conv_ldw<CIN>();
    constexpr int ROW16 = 27 * CIN * 2 / 16;  // 16-byte chunks per weight row
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __nv_bfloat16 *sW = reinterpret_cast<__nv_bfloat16 *>(smem_raw);
    for (int e = threadIdx.x; e < COUT * ROW16; e += blockDim.x) {
        const int o = e / ROW16, q = e % ROW16;
        reinterpret_cast<uint4 *>(sW + o * LDW)[q] = reinterpret_cast<const uint4 *>(W + (long long)o * 27 * CIN)[q];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, tg = lane & 3;
    const long long V = (long long)n * n * n;
    const long long v0 = ((long long)blockIdx.x * 4 + warp) * (MT * 16);
    if (v0 >= V) return;
    int zb[MT], yb[MT], xb[MT];
#pragma unroll
    for (int m = 0; m < MT; ++m) {
        const long long vb = v0 + 16 * m;
        zb[m] = (int)(vb % n);
        yb[m] = (int)((vb / n) % n);
        xb[m] = (int)(vb / ((long long)n * n));
    }
    float acc[MT][NT][4];
#pragma unroll
    for (int m = 0; m < MT; ++m)
#pragma unroll
        for (int j = 0; j < NT; ++j) acc[m][j][0] = acc[m][j][1] = acc[m][j][2] = acc[m][j][3] = 0.f;
    for (int t = 0; t < 27; ++t) {
        const __nv_bfloat16 *xa[MT], *xbp[MT];
#pragma unroll
        for (int m = 0; m < MT; ++m) {
            xa[m] = X + nbr(n, xb[m], yb[m], zb[m] + g, t) * CIN;
            xbp[m] = X + nbr(n, xb[m], yb[m], zb[m] + g + 8, t) * CIN;
        }
#pragma unroll
        for (int kc = 0; kc < CIN; kc += 16) {
            uint32_t a[MT][4];
#pragma unroll
            for (int m = 0; m < MT; ++m) {
                a[m][0] = ld_b32(xa[m] + kc + 2 * tg);
                a[m][1] = ld_b32(xbp[m] + kc + 2 * tg);
                a[m][2] = ld_b32(xa[m] + kc + 8 + 2 * tg);
                a[m][3] = ld_b32(xbp[m] + kc + 8 + 2 * tg);
            }
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                const __nv_bfloat16 *w = sW + (j * 8 + g) * LDW + t * CIN + kc + 2 * tg;
                const uint32_t b0 = ld_b32(w), b1 = ld_b32(w + 8);
#pragma unroll
                for (int m = 0; m < MT; ++m) mma_bf16(acc[m][j], a[m][0], a[m][1], a[m][2], a[m][3], b0, b1);
            }
        }
    }
#pragma unroll
    for (int m = 0; m < MT; ++m) {
#pragma unroll
        for (int j = 0; j < NT; ++j) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const long long v = v0 + 16 * m + g + 8 * h;
                const int o = j * 8 + 2 * tg;
                float y0 = acc[m][j][2 * h], y1 = acc[m][j][2 * h + 1];
                if (bias) {
                    y0 += bias[o];
                    y1 += bias[o + 1];
                }
                if constexpr (EPI == EPI_HIDDEN || EPI == EPI_OUT) {
                    Z[v * COUT + o] = y0;
                    Z[v * COUT + o + 1] = y1;
                }
                if constexpr (EPI == EPI_HIDDEN) {
                    *reinterpret_cast<__nv_bfloat162 *>(A + v * COUT + o) =
                        __floats2bfloat162_rn(gelu_f(y0), gelu_f(y1));
                }
                if constexpr (EPI == EPI_DGRAD) {
                    const float d0 = y0 * gelu_d(Zp[v * COUT + o]), d1 = y1 * gelu_d(Zp[v * COUT + o + 1]);
                    *reinterpret_cast<__nv_bfloat162 *>(A + v * COUT + o) = __floats2bfloat162_rn(d0, d1);
                }
            }
        }
    }
}

// Launch of one convolution layer (V / CONV_VOX blocks; V is a multiple of
// CONV_VOX for every supported n).
template <int CIN, int COUT, int EPI>
static cudaError_t conv(int n, const __nv_bfloat16 *X, const __nv_bfloat16 *W, const float *bias, float *Z,
                        __nv_bfloat16 *A, const float *Zp, cudaStream_t st) {
    const long long V = (long long)n * n * n;
    k_conv<CIN, COUT, EPI><<<(unsigned)((V + CONV_VOX - 1) / CONV_VOX), 128, conv_smem<CIN, COUT>(), st>>>(
        n, X, W, bias, Z, A, Zp);
    return cudaGetLastError();
}

template <int CIN, int COUT, int EPI> static cudaError_t conv_attr() {
    return cudaFuncSetAttribute(k_conv<CIN, COUT, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)conv_smem<CIN, COUT>());
}

// The same convolution on the fifth-generation tensor cores.  A block of
// 4 warps owns M = 128 consecutive voxels; the layer's weights (27 taps x
// CIN/16 K steps of COUT x 16 BF16, already in the core-matrix layout, see
// k_pack_canonical) sit in shared memory for the whole block.  For each tap
// the 128 threads gather their voxels' shifted activations (one row each,
// cp.async 16-byte copies) into one of NS A buffers in the core-matrix
// layout, NS - 2 taps ahead of the MMAs; one thread issues the tap's CIN/16
// MMAs (M 128, N COUT, K 16) accumulating in tensor memory and commits them
// to the buffer's mbarrier, and a buffer is refilled only after that commit
// (the MMAs of two taps back, so the wait for them is normally free).
// The accumulators are read back lane per voxel for the epilogues.  Every
// wait is bounded; on expiry the block records kErrWaitTimeout in *err,
// lets the issued MMAs finish (bounded) and frees its tensor memory.
template <int CIN, int COUT> struct ConvTc {
    static constexpr int KS = CIN / 16;          // K steps per tap
    static constexpr int BT = COUT / 8 * 256;    // bytes of one B tile (COUT x 16)
    static constexpr int BBYTES = 27 * KS * BT;  // all weights
    static constexpr int ABYTES = KS * 4096;     // one tap of A (128 x CIN)
    static constexpr int NS = 5;                 // A buffers (taps in flight)
    static constexpr size_t smem = (size_t)BBYTES + NS * ABYTES;
};

// W[o][t][c] (GPU layout, BF16) -> tiles (t, kk) of COUT x 16 in the K-major
// core-matrix layout: byte (o/8) 256 + (k/8) 128 + (o%8) 16 + (k%8) 2 of
// tile t KS + kk, k = c - 16 kk.
template <int CIN, int COUT>
__global__ void k_pack_canonical(const __nv_bfloat16 *__restrict__ W, __nv_bfloat16 *__restrict__ Wc) {
    typedef ConvTc<CIN, COUT> C;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= COUT * 27 * CIN) return;
    const int o = e / (27 * CIN), t = (e / CIN) % 27, c = e % CIN;
    const int kk = c / 16, k = c % 16;
    const int byte = (t * C::KS + kk) * C::BT + (o / 8) * 256 + (k / 8) * 128 + (o % 8) * 16 + (k % 8) * 2;
    Wc[byte / 2] = W[e];
}

__device__ __forceinline__ void cp_async16(void *dst_smem, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst_smem)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int PENDING> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(PENDING) : "memory");
}

template <int CIN, int COUT, int EPI>
__global__ void __launch_bounds__(128) k_conv_tc(int n, const __nv_bfloat16 *__restrict__ X,
                                                 const __nv_bfloat16 *__restrict__ Wc,
                                                 const float *__restrict__ bias, float *__restrict__ Z,
                                                 __nv_bfloat16 *__restrict__ A, const float *__restrict__ Zp,
                                                 int *err) {
    typedef ConvTc<CIN, COUT> C;
    constexpr int NS = C::NS;
    constexpr uint32_t IDESC = tc::idesc_bf16_f32(128, COUT);
    constexpr uint32_t TCOLS = 32;
    static_assert(COUT == 16 || COUT == 32, "one or two 16-column accumulator loads");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *sB = smem_raw;
    unsigned char *sA = smem_raw + C::BBYTES;
    __shared__ __align__(8) uint64_t bar[NS];
    __shared__ uint32_t tmem_base;
    __shared__ int s_ok;
    const int tid = threadIdx.x, warp = tid >> 5;
    const long long v = (long long)blockIdx.x * 128 + tid;  // this thread's voxel = row of the M tile
    const int z = (int)(v % n), y = (int)((v / n) % n), x = (int)(v / ((long long)n * n));
    // this thread's row in an A buffer (chunk c of 8 channels at + (c/2) 4096 + (c%2) 128)
    unsigned char *arow = sA + (tid / 8) * 256 + (tid % 8) * 16;
    auto gather = [&](int t) {  // cp.async of tap t into buffer t % NS, one commit group
        const __nv_bfloat16 *src = X + nbr(n, x, y, z, t) * CIN;
        unsigned char *dst = arow + (t % NS) * C::ABYTES;
#pragma unroll
        for (int c = 0; c < CIN / 8; ++c) cp_async16(dst + (c / 2) * 4096 + (c % 2) * 128, src + 8 * c);
        cp_async_commit();
    };
#pragma unroll
    for (int t = 0; t < NS - 2; ++t) gather(t);
    for (int e = tid; e < C::BBYTES / 16; e += 128)
        reinterpret_cast<uint4 *>(sB)[e] = reinterpret_cast<const uint4 *>(Wc)[e];
    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < NS; ++i) mbar_init(&bar[i], 1);
        s_ok = 1;
    }
    if (warp == 0) tc::tmem_alloc(&tmem_base, TCOLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tmem_base;
    int issued = -1;  // last tap whose MMAs were committed (thread 0)
    for (int t = 0; t < 27; ++t) {
        // refill buffer (t + NS - 2) % NS, last read by the MMAs of tap t - 2
        const int tn = t + NS - 2;
        if (tn < 27) {
            if (t >= 2) {
                if (tid == 0) s_ok = mbar_wait_bounded(&bar[(t - 2) % NS], ((t - 2) / NS) & 1) ? 1 : 0;
                __syncthreads();
                if (!s_ok) break;
            }
            gather(tn);
        } else {
            cp_async_commit();  // an empty group keeps the count of pending groups fixed
        }
        cp_async_wait<NS - 2>();  // this thread's copies of tap t have landed
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const unsigned char *a = sA + (t % NS) * C::ABYTES;
#pragma unroll
            for (int kk = 0; kk < C::KS; ++kk)
                tc::mma_bf16(taddr, tc::smem_desc(a + kk * 4096, 128, 256),
                             tc::smem_desc(sB + (t * C::KS + kk) * C::BT, 128, 256), IDESC, t > 0 || kk > 0);
            tc::commit(&bar[t % NS]);
            issued = t;
        }
    }
    cp_async_wait<0>();
    if (tid == 0) {  // the commit of the last issued tap covers every earlier MMA
        const bool done = issued < 0 || mbar_wait_bounded(&bar[issued % NS], (issued / NS) & 1);
        if (!done || !s_ok || issued != 26) {
            s_ok = 0;
            record_error(err, kErrWaitTimeout);
        }
    }
    __syncthreads();
    tc::fence_after_sync();
    if (s_ok) {
        float acc[COUT];
        tc::ld16(taddr + ((uint32_t)(32 * warp) << 16), *reinterpret_cast<float(*)[16]>(acc));
        if constexpr (COUT == 32)
            tc::ld16(taddr + ((uint32_t)(32 * warp) << 16) + 16, *reinterpret_cast<float(*)[16]>(acc + 16));
#pragma unroll
        for (int o = 0; o < COUT; o += 2) {
            float y0 = acc[o], y1 = acc[o + 1];
            if (bias) {
                y0 += bias[o];
                y1 += bias[o + 1];
            }
            if constexpr (EPI == EPI_HIDDEN || EPI == EPI_OUT) {
                *reinterpret_cast<float2 *>(Z + v * COUT + o) = make_float2(y0, y1);
            }
            if constexpr (EPI == EPI_HIDDEN) {
                *reinterpret_cast<__nv_bfloat162 *>(A + v * COUT + o) = __floats2bfloat162_rn(gelu_f(y0), gelu_f(y1));
            }
            if constexpr (EPI == EPI_DGRAD) {
                const float2 zp = *reinterpret_cast<const float2 *>(Zp + v * COUT + o);
                *reinterpret_cast<__nv_bfloat162 *>(A + v * COUT + o) =
                    __floats2bfloat162_rn(y0 * gelu_d(zp.x), y1 * gelu_d(zp.y));
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, TCOLS);
}

template <int CIN, int COUT, int EPI>
static cudaError_t conv_tc(int n, const __nv_bfloat16 *X, const __nv_bfloat16 *Wc, const float *bias, float *Z,
                           __nv_bfloat16 *A, const float *Zp, int *err, cudaStream_t st) {
    const long long V = (long long)n * n * n;
    k_conv_tc<CIN, COUT, EPI><<<(unsigned)(V / 128), 128, ConvTc<CIN, COUT>::smem, st>>>(n, X, Wc, bias, Z, A, Zp,
                                                                                          err);
    return cudaGetLastError();
}

template <int CIN, int COUT, int EPI> static cudaError_t conv_tc_attr() {
    return cudaFuncSetAttribute(k_conv_tc<CIN, COUT, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)ConvTc<CIN, COUT>::smem);
}

// The same convolution on the fifth-generation tensor cores, fed from a
// shared-memory halo slab instead of per-tap gathers.  A persistent block
// walks work items (x, y0): Y consecutive z lines (x, y0 .. y0+Y-1).  For an
// item it lands, by 16-byte cp.async copies (one warp per line), the slab of
// input rows x-1..x+1, y0-1..y0+Y and z = -1..n (periodic), one row per
// voxel, in the K-major core-matrix layout [CIN/8 chunks][rows][8 BF16] with
// the rows of a z line consecutive:
//   slab row s = (xi (Y+2) + yi) (n+2) + r,  xi, yi, r = x, y, z offsets + 1.
// Output positions p = yl (n+2) + r run over the item's lines with their
// two halo rows (invalid outputs, never stored).  The input of tap
// (dx, dy, dz) for output p is slab row p + (1+dx)(Y+2)(n+2) + (1+dy)(n+2)
// + dz, a fixed shift for all p: each tap's A operand of an M = 128 tile of
// positions is the same slab read from a shifted start address, so the 27
// taps' MMAs (CIN/16 K steps each) of every tile are issued back to back
// with no gather or barrier between them.  The layer's weights (27 CIN/16
// tiles of COUT x 16) stay in shared memory for the whole block.
//
// Roles: warp 0 issues the MMAs (one thread), warps 1..4 copy slabs, warps
// 5..12 run the epilogue (two groups, each covering the four quadrants of the
// 128 tensor-memory lanes, taking alternate (tile, 16-channel) units), so the
// copies of item j + 1, the MMAs of item j and the epilogue of item j - 1
// overlap.  The epilogue reads 16 accumulator columns of its 32 rows at a
// time and passes them through a per-warp shared-memory stage, so global
// stores (and the loads of the forward pre-activations a gradient layer
// needs) move whole 16-byte pieces of consecutive voxels rather than one
// 8-byte piece per voxel and lane.
// Hand-offs are mbarriers:
//   slab_full[b]  copy warps -> MMA warp: slab buffer b has landed
//   mma_done[a]   MMA commit -> copy warps: the item's slab buffer is free;
//                 -> epilogue warps: accumulator a is readable
//   acc_free[a]   epilogue warps -> MMA warp: accumulator a has been read
// Two slab buffers (one where two do not fit) and two accumulators let the
// copies of the next item and the epilogue of the previous one run while
// the current item's MMAs execute.  Every wait is bounded; on expiry the
// waiting thread records kErrWaitTimeout, every role leaves its loop at its
// next check, the issued MMAs are waited for (bounded) and the tensor
// memory is freed.
struct SlabGeom {
    int n, Y, rows, tiles, nbuf;
    size_t slab_bytes, smem;
};

template <int CIN, int COUT> struct ConvSlab {
    static constexpr int KS = CIN / 16;         // K steps per tap
    static constexpr int CH = CIN / 8;          // 16-byte chunks per voxel row
    static constexpr int BT = COUT / 8 * 256;   // bytes of one B tile (COUT x 16)
    static constexpr int BBYTES = 27 * KS * BT; // all weights
    static constexpr int ACC_COLS = 128;        // tensor-memory columns per accumulator buffer
    // epilogue staging per warp: 32 rows x 16 channels of FP32 (rows of 20),
    // reused for the same rows in BF16 (rows of 24), so results leave in
    // 16-byte pieces
    static constexpr int ZLD = 20, ALD = 24;
    static constexpr int STAGE_WARP = 32 * ZLD * 4;
    static constexpr int STAGE_BYTES = 8 * STAGE_WARP;  // eight epilogue warps
    static SlabGeom geom(int n) {
        SlabGeom g{};
        g.n = n;
        g.Y = n <= 16 ? 8 : (n <= 64 ? 4 : 1);
        if (g.Y > n) g.Y = n;
        g.rows = 3 * (g.Y + 2) * (n + 2) + 2;  // + one padding row at each end
        g.tiles = (g.Y * (n + 2) + 127) / 128;
        g.slab_bytes = (size_t)CH * g.rows * 16;
        const size_t fixed = (size_t)BBYTES + STAGE_BYTES;
        g.nbuf = fixed + 2 * g.slab_bytes <= kMaxSmemLes ? 2 : 1;
        // at least 80 KB, so no more than two blocks share an SM: each holds
        // 256 of the SM's 512 tensor-memory columns
        g.smem = fixed + g.nbuf * g.slab_bytes;
        if (g.smem < 80 * 1024) g.smem = 80 * 1024;
        return g;
    }
};

constexpr int kSlabCopyWarps = 4;  // warps 1..4 land the slabs
constexpr int kSlabEpiWarps = 8;   // warps 5..12 read the accumulators (two per tensor-memory lane quadrant)
constexpr int kSlabThreads = 32 * (1 + kSlabCopyWarps + kSlabEpiWarps);  // + the MMA warp (0)

// Bounded mbarrier wait; on expiry marks the block failed (shared flag) and
// records the timeout.  Returns false if the block has failed.
__device__ __forceinline__ bool slab_wait(uint64_t *bar, uint32_t parity, volatile int *ok, int *err) {
    if (!*ok) return false;
    if (mbar_wait_bounded(bar, parity)) return true;
    *ok = 0;
    record_error(err, kErrWaitTimeout);
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

template <int CIN, int COUT, int EPI>
__global__ void __launch_bounds__(kSlabThreads, 1) k_conv_slab(SlabGeom sg, const __nv_bfloat16 *__restrict__ X,
                                                              const __nv_bfloat16 *__restrict__ Wc,
                                                              const float *__restrict__ bias, float *__restrict__ Z,
                                                              __nv_bfloat16 *__restrict__ A,
                                                              const float *__restrict__ Zp, int *err) {
    typedef ConvSlab<CIN, COUT> C;
    constexpr uint32_t IDESC = tc::idesc_bf16_f32(128, COUT);
    constexpr uint32_t TCOLS = 2 * C::ACC_COLS;
    constexpr int NCOPY = 32 * kSlabCopyWarps, NEPI = 32 * kSlabEpiWarps;
    static_assert(COUT == 16 || COUT == 32, "one or two 16-column accumulator loads");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *sB = smem_raw;
    unsigned char *sSlab = smem_raw + C::BBYTES;
    __shared__ __align__(8) uint64_t slab_full[2], mma_done[2], acc_free[2];
    __shared__ uint32_t tmem_base;
    __shared__ volatile int s_ok;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n = sg.n, Y = sg.Y, L = n + 2, rows = sg.rows;
    const int plane = (Y + 2) * L;  // slab rows per x plane
    const int ybl = n / Y;          // items per x plane
    const long long items = (long long)n * ybl;
    const int nbuf = sg.nbuf;

    for (int e = tid; e < C::BBYTES / 16; e += kSlabThreads)
        reinterpret_cast<uint4 *>(sB)[e] = reinterpret_cast<const uint4 *>(Wc)[e];
    fence_proxy_async_smem();  // the weights are read by the MMAs (async proxy)
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&slab_full[i], NCOPY);
            mbar_init(&mma_done[i], 1);
            mbar_init(&acc_free[i], NEPI);
        }
        s_ok = 1;
    }
    if (warp == 0) tc::tmem_alloc(&tmem_base, TCOLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const long long first = blockIdx.x, stride = gridDim.x;
    const int nitems = first < items ? (int)((items - 1 - first) / stride + 1) : 0;

    if (warp == 0) {
        // ---------------- MMA warp: one thread issues, the warp stays converged
        int committed = -1;
        if (lane == 0) {
            const uint32_t lbo16 = (uint32_t)rows;  // K-adjacent core matrices: next chunk (rows x 16 B) >> 4
            const uint64_t bdesc0 = tc::smem_desc(sB, 128, 256);
            const int npos = Y * L;
            for (int j = 0; j < nitems; ++j) {
                const int b = nbuf == 2 ? (j & 1) : 0;
                const uint32_t ub = nbuf == 2 ? (uint32_t)(j >> 1) : (uint32_t)j;  // uses of slab buffer b
                if (!slab_wait(&slab_full[b], ub & 1, &s_ok, err)) break;
                if (j >= 2 && !slab_wait(&acc_free[j & 1], (uint32_t)(((j - 2) >> 1) & 1), &s_ok, err)) break;
                tc::fence_after_sync();
                // A descriptor of slab row 0 of buffer b (after the front padding row)
                const uint32_t a0 = smem_addr(sSlab + (size_t)b * sg.slab_bytes) + 16;
                const uint64_t adesc0 = (uint64_t)((a0 & 0x3FFFFu) >> 4) | ((uint64_t)(lbo16 & 0x3FFFu) << 16) |
                                        ((uint64_t)(128 >> 4) << 32) | (1ull << 46);
                const uint32_t tacc = tmem_base + (uint32_t)((j & 1) * C::ACC_COLS);
                // tile by tile, all 27 taps' MMAs back to back (a single thread's
                // descriptor arithmetic stays in registers: a runtime-indexed
                // array here would be reloaded from local memory after every
                // MMA, whose asm is a compiler memory barrier)
                for (int t = 0; t < sg.tiles; ++t) {
                    const int p0 = min(128 * t, npos - 128);
#pragma unroll
                    for (int tap = 0; tap < 27; ++tap) {
                        const int dx = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dz = tap % 3 - 1;
                        // slab row of output p0 for this tap, in 16-byte units (-1 for
                        // the first tap of the first tile: the front padding row);
                        // signed, so the sum with the descriptor's address field
                        // never borrows
                        const int row = p0 + dz + (1 + dx) * plane + (1 + dy) * L;
#pragma unroll
                        for (int kk = 0; kk < C::KS; ++kk) {
                            const uint64_t adesc = (uint64_t)((long long)adesc0 + (long long)(row + 2 * kk * rows));
                            const uint64_t bdesc = bdesc0 + (uint64_t)(((tap * C::KS + kk) * C::BT) >> 4);
                            tc::mma_bf16(tacc + t * COUT, adesc, bdesc, IDESC, tap > 0 || kk > 0);
                        }
                    }
                }
                tc::commit(&mma_done[j & 1]);
                committed = j;
            }
            if (!s_ok && committed >= 0)  // let the issued MMAs finish before the memory is freed
                mbar_wait_bounded(&mma_done[committed & 1], (uint32_t)((committed >> 1) & 1));
        }
        __syncwarp();
    } else if (warp <= kSlabCopyWarps) {
        // ---------------- copy warps: one slab line per warp at a time; its n
        // voxels are contiguous in X, lane e copies chunk e mod CH of row
        // e / CH (the halo rows r = 0 and r = n + 1 wrap to z = n - 1, 0)
        const int cw = warp - 1;
        for (int j = 0; j < nitems; ++j) {
            const int b = nbuf == 2 ? (j & 1) : 0;
            const int jb = j - nbuf;  // the buffer was last read by the MMAs of item jb
            if (jb >= 0 && !slab_wait(&mma_done[jb & 1], (uint32_t)((jb >> 1) & 1), &s_ok, err)) break;
            const long long w = first + (long long)j * stride;
            const int x = (int)(w / ybl), y0 = (int)(w % ybl) * Y;
            unsigned char *dst = sSlab + (size_t)b * sg.slab_bytes;
            const int nlines = 3 * (Y + 2);
            for (int li = cw; li < nlines; li += kSlabCopyWarps) {
                const int xi = li / (Y + 2), yi = li % (Y + 2);
                const int gx = (x - 1 + xi + n) % n, gy = (y0 - 1 + yi + n) % n;
                const __nv_bfloat16 *src = X + ((long long)gx * n + gy) * n * CIN;
                unsigned char *d = dst + ((size_t)li * L + 1) * 16;  // + the front padding row
                for (int e = lane; e < L * C::CH; e += 32) {
                    const int r = e / C::CH, c = e % C::CH;
                    const int z = r == 0 ? n - 1 : (r == n + 1 ? 0 : r - 1);
                    cp_async16(d + ((size_t)c * rows + r) * 16, src + (long long)z * CIN + 8 * c);
                }
            }
            cp_async_commit();
            cp_async_wait<0>();
            fence_proxy_async_smem();
            mbar_arrive(&slab_full[b]);
        }
        cp_async_wait<0>();
    } else {
        // ---------------- epilogue warps
        const int ew = warp - 1 - kSlabCopyWarps;  // 0..7
        const int wq = warp & 3;                   // tensor-memory lane quadrant this warp may read
        const int grp = ew >> 2;                   // units u = grp, grp + 2, ...
        float *zst = reinterpret_cast<float *>(sSlab + (size_t)nbuf * sg.slab_bytes + (size_t)ew * C::STAGE_WARP);
        __nv_bfloat16 *ast = reinterpret_cast<__nv_bfloat16 *>(zst);  // the same rows, later, in BF16
        const int npos = Y * L;
        constexpr int HALVES = COUT / 16;
        for (int j = 0; j < nitems; ++j) {
            if (!slab_wait(&mma_done[j & 1], (uint32_t)((j >> 1) & 1), &s_ok, err)) break;
            tc::fence_after_sync();
            const long long w = first + (long long)j * stride;
            const int x = (int)(w / ybl), y0 = (int)(w % ybl) * Y;
            const uint32_t tacc = tmem_base + (uint32_t)((j & 1) * C::ACC_COLS) + ((uint32_t)(32 * wq) << 16);
            for (int u = grp; u < sg.tiles * HALVES; u += 2) {
                const int t = u / HALVES, h = u % HALVES;
                const int p0 = min(128 * t, npos - 128);
                // this lane's row: its voxel, or -1 (halo row, or a row the
                // previous tile already produced); other rows' by shuffle
                long long vme;
                {
                    const int p = p0 + 32 * wq + lane;
                    const int yl = p / L, z = p % L - 1;
                    vme = (p < 128 * t || z < 0 || z >= n) ? -1 : ((long long)x * n + (y0 + yl)) * n + z;
                }
                float acc[16];
                tc::ld16(tacc + t * COUT + 16 * h, acc);
                float zp[16];
                if constexpr (EPI == EPI_DGRAD) {
                    // forward pre-activations of these rows and channels, staged
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int e = lane + 32 * k, r = e >> 2, q = e & 3;
                        const long long v = __shfl_sync(0xffffffffu, vme, r);
                        float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (v >= 0) z4 = *reinterpret_cast<const float4 *>(Zp + v * COUT + 16 * h + 4 * q);
                        *reinterpret_cast<float4 *>(zst + r * C::ZLD + 4 * q) = z4;
                    }
                    __syncwarp();
#pragma unroll
                    for (int o = 0; o < 16; ++o) zp[o] = zst[lane * C::ZLD + o];
                    __syncwarp();
                }
                float yv[16];
#pragma unroll
                for (int o = 0; o < 16; ++o) yv[o] = acc[o] + (bias ? bias[16 * h + o] : 0.f);
                if constexpr (EPI == EPI_HIDDEN || EPI == EPI_OUT) {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        *reinterpret_cast<float4 *>(zst + lane * C::ZLD + 4 * q) =
                            make_float4(yv[4 * q], yv[4 * q + 1], yv[4 * q + 2], yv[4 * q + 3]);
                    __syncwarp();
                    // whole 16-byte pieces out, 4 lanes per row
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int e = lane + 32 * k, r = e >> 2, q = e & 3;
                        const long long v = __shfl_sync(0xffffffffu, vme, r);
                        if (v >= 0)
                            *reinterpret_cast<float4 *>(Z + v * COUT + 16 * h + 4 * q) =
                                *reinterpret_cast<const float4 *>(zst + r * C::ZLD + 4 * q);
                    }
                    __syncwarp();
                }
                if constexpr (EPI == EPI_HIDDEN || EPI == EPI_DGRAD) {
                    __nv_bfloat162 a2[8];
#pragma unroll
                    for (int o = 0; o < 16; o += 2) {
                        if constexpr (EPI == EPI_HIDDEN)
                            a2[o / 2] = __floats2bfloat162_rn(gelu_f(yv[o]), gelu_f(yv[o + 1]));
                        else
                            a2[o / 2] = __floats2bfloat162_rn(yv[o] * gelu_d(zp[o]), yv[o + 1] * gelu_d(zp[o + 1]));
                    }
                    uint4 *ad = reinterpret_cast<uint4 *>(ast + lane * C::ALD);
                    ad[0] = *reinterpret_cast<const uint4 *>(&a2[0]);
                    ad[1] = *reinterpret_cast<const uint4 *>(&a2[4]);
                    __syncwarp();
                    // whole 16-byte pieces out, 2 lanes per row
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        const int e = lane + 32 * k, r = e >> 1, q = e & 1;
                        const long long v = __shfl_sync(0xffffffffu, vme, r);
                        if (v >= 0)
                            *reinterpret_cast<uint4 *>(A + v * COUT + 16 * h + 8 * q) =
                                *reinterpret_cast<const uint4 *>(ast + r * C::ALD + 8 * q);
                    }
                    __syncwarp();
                }
            }
            tc::fence_before_sync();
            mbar_arrive(&acc_free[j & 1]);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem_base, TCOLS);
}

template <int CIN, int COUT, int EPI>
static cudaError_t conv_slab(int n, const __nv_bfloat16 *X, const __nv_bfloat16 *Wc, const float *bias, float *Z,
                             __nv_bfloat16 *A, const float *Zp, int *err, cudaStream_t st) {
    const SlabGeom g = ConvSlab<CIN, COUT>::geom(n);
    if (g.Y * (n + 2) < 128 || g.tiles * COUT > ConvSlab<CIN, COUT>::ACC_COLS || g.smem > kMaxSmemLes)
        return cudaErrorInvalidValue;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const long long items = (long long)n * (n / g.Y);
    const unsigned grid = (unsigned)(items < sms ? items : sms);
    k_conv_slab<CIN, COUT, EPI><<<grid, kSlabThreads, g.smem, st>>>(g, X, Wc, bias, Z, A, Zp, err);
    return cudaGetLastError();
}

template <int CIN, int COUT, int EPI> static cudaError_t conv_slab_attr() {
    return cudaFuncSetAttribute(k_conv_slab<CIN, COUT, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kMaxSmemLes);
}

// Weight gradient partials: block (chunk, tap) accumulates
// D[o][c] = sum_{v in chunk} dY[v][o] X[v + off(t)][c] (M = COUTP rows o,
// N = CIN cols c, K = voxels) and writes it to P[chunk][t][o][c].  COUTP is
// COUT rounded up to 16 (the MMA's M); the extra rows are zero.
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) k_wgrad(int n, const __nv_bfloat16 *__restrict__ dY,
                                               const __nv_bfloat16 *__restrict__ X, float *__restrict__ P,
                                               int chunk) {
    constexpr int COUTP = COUT < 16 ? 16 : COUT;
    constexpr int MT = COUTP / 16, NT = CIN / 8;
    constexpr int SUB = 128;  // voxels staged per round
    constexpr int LDA = SUB + 8, LDB = SUB + 8;  // padded rows (bank spread)
    __shared__ __align__(16) __nv_bfloat16 sA[COUTP * LDA];
    __shared__ __align__(16) __nv_bfloat16 sB[CIN * LDB];
    const int t = blockIdx.y;
    const long long V = (long long)n * n * n;
    const long long vbeg = (long long)blockIdx.x * chunk;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, tg = lane & 3;
    // warps own (m-tile, n-tile) pairs round robin
    constexpr int TILES = MT * NT;
    float acc[(TILES + 7) / 8][4];
#pragma unroll
    for (int i = 0; i < (TILES + 7) / 8; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
    for (long long vs = vbeg; vs < vbeg + chunk && vs < V; vs += SUB) {
        __syncthreads();
        for (int e = threadIdx.x; e < SUB * COUTP; e += blockDim.x) {
            const int v = e / COUTP, o = e % COUTP;
            const long long vv = vs + v;
            sA[o * LDA + v] = (o < COUT && vv < V) ? dY[vv * COUT + o] : __float2bfloat16(0.f);
        }
        for (int e = threadIdx.x; e < SUB * CIN; e += blockDim.x) {
            const int v = e / CIN, c = e % CIN;
            const long long vv = vs + v;
            __nv_bfloat16 val = __float2bfloat16(0.f);
            if (vv < V) {
                const int z = (int)(vv % n), y = (int)((vv / n) % n), x = (int)(vv / ((long long)n * n));
                val = X[nbr(n, x, y, z, t) * CIN + c];
            }
            sB[c * LDB + v] = val;
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < (TILES + 7) / 8; ++i) {
            const int tile = warp + 8 * i;
            if (tile < TILES) {
                const int mt = tile / NT, nt = tile % NT;
                for (int k = 0; k < SUB; k += 16) {
                    const __nv_bfloat16 *a = sA + (mt * 16 + g) * LDA + k + 2 * tg;
                    const __nv_bfloat16 *b = sB + (nt * 8 + g) * LDB + k + 2 * tg;
                    mma_bf16(acc[i], ld_b32(a), ld_b32(a + 8 * LDA), ld_b32(a + 8), ld_b32(a + 8 * LDA + 8),
                             ld_b32(b), ld_b32(b + 8));
                }
            }
        }
    }
    float *out = P + ((long long)blockIdx.x * 27 + t) * COUT * CIN;
#pragma unroll
    for (int i = 0; i < (TILES + 7) / 8; ++i) {
        const int tile = warp + 8 * i;
        if (tile < TILES) {
            const int mt = tile / NT, nt = tile % NT;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int o = mt * 16 + g + 8 * h, c = nt * 8 + 2 * tg;
                if (o < COUT) {
                    out[o * CIN + c] = acc[i][2 * h];
                    out[o * CIN + c + 1] = acc[i][2 * h + 1];
                }
            }
        }
    }
}

// sum over chunks in a fixed order: G[o][t][c] (GPU layout) += sum_b P[b][t][o][c]
__global__ void k_wgrad_reduce(const float *__restrict__ P, int nchunk, int cout, int cin, float *__restrict__ G) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int total = 27 * cout * cin;
    if (e >= total) return;
    const int t = e / (cout * cin), o = (e / cin) % cout, c = e % cin;
    float s = 0.f;
    for (int b = 0; b < nchunk; ++b) s += P[((long long)b * 27 + t) * cout * cin + o * cin + c];
    G[((long long)o * 27 + t) * cin + c] += s;
}

// column sums of a [V][C] BF16 array into G (bias gradient), fixed order
__global__ void k_colsum(const __nv_bfloat16 *__restrict__ d, long long V, int C, int creal, float *__restrict__ G) {
    __shared__ float red[256];
    const int c = blockIdx.x;
    float s = 0.f;
    for (long long v = threadIdx.x; v < V; v += blockDim.x) s += __bfloat162float(d[v * C + c]);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0 && c < creal) G[c] += red[0];
}

// g[9][V] floats -> X0[V][16] BF16 (channels 9..15 zero)
// One thread per voxel: nine reads, each coalesced along v, and the voxel's
// 32-byte row written as two 16-byte stores.
__global__ void k_prep_input(const float *__restrict__ g, long long V, __nv_bfloat16 *__restrict__ X0) {
    const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= V) return;
    __align__(16) __nv_bfloat16 row[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) row[c] = __float2bfloat16(c < 9 ? g[c * V + v] : 0.f);
    uint4 *dst = reinterpret_cast<uint4 *>(X0 + v * 16);
    dst[0] = reinterpret_cast<const uint4 *>(row)[0];
    dst[1] = reinterpret_cast<const uint4 *>(row)[1];
}

// The output layer is computed 16 channels wide (the MMA's K granularity for
// its input gradient); channels 6..15 are zero.
constexpr int OUTP = 16;

// MSE: dY[v][o] = 2 (Y - tau) / (6 V) (BF16, o < 6; padding zero), per-block partial loss
__global__ void k_mse(const float *__restrict__ Y, const float *__restrict__ tau, long long V,
                      __nv_bfloat16 *__restrict__ dY, double *__restrict__ partial) {
    __shared__ double red[256];
    double s = 0.0;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
        for (int o = 0; o < OUTP; ++o) {
            float d = 0.f;
            if (o < 6) {
                d = Y[v * OUTP + o] - tau[o * V + v];
                s += (double)d * d;
            }
            dY[v * OUTP + o] = __float2bfloat16(2.0f * d / (6.0f * (float)V));
        }
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_sum_d(const double *p, int n, double scale, double *out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += p[i];
        *out += s * scale;
    }
}

// Y[V][OUTP] -> tau[6][V] floats
// One thread per voxel: the first six channels of its row (one 16-byte and
// one 8-byte load) to the six planes of tau, each store coalesced along v.
__global__ void k_out_to_tau(const float *__restrict__ Y, long long V, float *__restrict__ tau, float scale) {
    const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (v >= V) return;
    const float4 a = *reinterpret_cast<const float4 *>(Y + v * OUTP);
    const float2 b = *reinterpret_cast<const float2 *>(Y + v * OUTP + 4);
    tau[v] = scale * a.x;
    tau[V + v] = scale * a.y;
    tau[2 * V + v] = scale * a.z;
    tau[3 * V + v] = scale * a.w;
    tau[4 * V + v] = scale * b.x;
    tau[5 * V + v] = scale * b.y;
}

// The output layer's six biases padded with zeros to its sixteen computed
// channels, so every engine's epilogue adds them like a hidden layer's.
__global__ void k_pad_bias(const float *__restrict__ b, int n, float *__restrict__ bp, int np) {
    const int i = threadIdx.x;
    if (i < np) bp[i] = i < n ? b[i] : 0.f;
}

// Master FP32 parameters in the oracle's layout ([Cout][Cin][27] weights)
// -> BF16 padded [Coutp][27][Cinp] and the flipped transpose used for input
// gradients, Wf[c][t][o] = W[o][26 - t][c] (padded to [Cinp... as Cout of the
// transposed convolution][27][Coutp]).
__global__ void k_pack_weights(const float *__restrict__ w, int cout, int cin, int coutp, int cinp,
                               __nv_bfloat16 *__restrict__ Wp, __nv_bfloat16 *__restrict__ Wf) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= coutp * 27 * cinp) return;
    const int o = e / (27 * cinp), t = (e / cinp) % 27, c = e % cinp;
    const float v = (o < cout && c < cin) ? w[((long long)o * cin + c) * 27 + t] : 0.f;
    Wp[e] = __float2bfloat16(v);
    if (Wf) Wf[((long long)c * 27 + (26 - t)) * coutp + o] = __float2bfloat16(v);
}

// Adam on the master parameters; gradients of weights come in the GPU layout
// [Coutp][27][Cinp] (gw_layout = 1) or are flat (biases, gw_layout = 0).
__global__ void k_adam(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ gsrc, int count, int gw_layout, int cout, int cin, int cinp,
                       float lr, float b1, float b2, float eps, float c1, float c2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count) return;
    float gr;
    if (gw_layout) {
        const int o = e / (cin * 27), c = (e / 27) % cin, t = e % 27;
        gr = gsrc[((long long)o * 27 + t) * cinp + c];
    } else {
        gr = gsrc[e];
    }
    const float mm = b1 * m[e] + (1.f - b1) * gr;
    const float vv = b2 * v[e] + (1.f - b2) * gr * gr;
    m[e] = mm;
    v[e] = vv;
    p[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

}  // namespace les
}  // namespace dns

using namespace dns::les;

// ---------------------------------------------------------------- network object
struct dns_net_ctx {
    int n = 0;  // mesh the buffers are sized for
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // master parameters (oracle layout), Adam moments, gradients
    float *p = nullptr, *m = nullptr, *v = nullptr;
    float *gw1 = nullptr, *gw2 = nullptr, *gw3 = nullptr, *gb = nullptr;  // GPU-layout weight grads; bias grads
    long step = 0;
    // BF16 packed weights, and the same in the tensor-core operand layout
    __nv_bfloat16 *W1 = nullptr, *W2 = nullptr, *W3 = nullptr, *W2f = nullptr, *W3f = nullptr;
    __nv_bfloat16 *W1c = nullptr, *W2c = nullptr, *W3c = nullptr, *W2fc = nullptr, *W3fc = nullptr;
    int *err = nullptr;  // device status word of the convolutions' bounded waits
    int engine = DNS_CONV_TCGEN05_SLAB;  // convolution engine (dns_conv_engine); the fastest is the default
    // activations for one sample
    __nv_bfloat16 *X0 = nullptr, *A1 = nullptr, *A2 = nullptr, *dY3 = nullptr, *dZ2 = nullptr, *dZ1 = nullptr;
    float *Z1 = nullptr, *Z2 = nullptr, *Y3 = nullptr, *wpart = nullptr;
    float *b3p = nullptr;  // output biases padded to OUTP (zeros beyond the six)
    double *lpart = nullptr, *lsum = nullptr, *hostd = nullptr;
    int nchunk = 0;
    float in_scale = 1.f, out_scale = 1.f;  // closure use: input g * in_scale, tau = output * out_scale
};

// parameter blocks in the flat master vector
static const long NET_W1 = 32L * 9 * 27, NET_B1 = 32, NET_W2 = 32L * 32 * 27, NET_B2 = 32, NET_W3 = 6L * 32 * 27,
                  NET_B3 = 6;
static const long OFF_W1 = 0, OFF_B1 = OFF_W1 + NET_W1, OFF_W2 = OFF_B1 + NET_B1, OFF_B2 = OFF_W2 + NET_W2,
                  OFF_W3 = OFF_B2 + NET_B2, OFF_B3 = OFF_W3 + NET_W3, NET_PARAMS = OFF_B3 + NET_B3;

static void net_release(dns_net_ctx *c) {
    if (!c) return;
    void *bufs[] = {c->p,   c->m,   c->v,    c->gw1,  c->gw2,  c->gw3, c->gb,  c->W1,  c->W2,    c->W3,
                    c->W2f, c->W3f, c->W1c,  c->W2c,  c->W3c,  c->W2fc, c->W3fc, c->err, c->X0,   c->A1,
                    c->A2,  c->dY3, c->dZ2,  c->dZ1,  c->Z1,   c->Z2,  c->Y3,  c->wpart, c->lpart, c->lsum, c->b3p};
    for (void *b : bufs)
        if (b) cudaFree(b);
    if (c->hostd) cudaFreeHost(c->hostd);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

static cudaError_t net_pack(dns_net_ctx *c) {
    k_pack_weights<<<nblk(32 * 27 * 16), 256, 0, c->stream>>>(c->p + OFF_W1, 32, 9, 32, 16, c->W1, nullptr);
    k_pack_weights<<<nblk(32 * 27 * 32), 256, 0, c->stream>>>(c->p + OFF_W2, 32, 32, 32, 32, c->W2, c->W2f);
    k_pack_weights<<<nblk(OUTP * 27 * 32), 256, 0, c->stream>>>(c->p + OFF_W3, 6, 32, OUTP, 32, c->W3, c->W3f);
    k_pack_canonical<16, 32><<<nblk(32 * 27 * 16), 256, 0, c->stream>>>(c->W1, c->W1c);
    k_pack_canonical<32, 32><<<nblk(32 * 27 * 32), 256, 0, c->stream>>>(c->W2, c->W2c);
    k_pack_canonical<32, OUTP><<<nblk(OUTP * 27 * 32), 256, 0, c->stream>>>(c->W3, c->W3c);
    k_pack_canonical<32, 32><<<nblk(32 * 27 * 32), 256, 0, c->stream>>>(c->W2f, c->W2fc);
    k_pack_canonical<OUTP, 32><<<nblk(32 * 27 * OUTP), 256, 0, c->stream>>>(c->W3f, c->W3fc);
    k_pad_bias<<<1, 32, 0, c->stream>>>(c->p + OFF_B3, (int)NET_B3, c->b3p, OUTP);
    return cudaGetLastError();
}

// forward of one sample already in X0; leaves Z1, A1, Z2, A2, Y3
// One convolution layer on the network's engine; W is the GPU-layout
// weight array, Wc the same in the tensor-core operand layout.
template <int CIN, int COUT, int EPI>
static cudaError_t conv_layer(dns_net_ctx *c, const __nv_bfloat16 *X, const __nv_bfloat16 *W,
                              const __nv_bfloat16 *Wc, const float *bias, float *Z, __nv_bfloat16 *A, const float *Zp,
                              cudaStream_t st) {
    if (c->engine == DNS_CONV_TCGEN05) return conv_tc<CIN, COUT, EPI>(c->n, X, Wc, bias, Z, A, Zp, c->err, st);
    if (c->engine == DNS_CONV_TCGEN05_SLAB)
        return conv_slab<CIN, COUT, EPI>(c->n, X, Wc, bias, Z, A, Zp, c->err, st);
    return conv<CIN, COUT, EPI>(c->n, X, W, bias, Z, A, Zp, st);
}

// The three layers from X0; with ev (4 events) recorded before the first
// layer and after each one, on st.
static cudaError_t net_forward_x0(dns_net_ctx *c, cudaStream_t st, cudaEvent_t *ev = nullptr) {
    cudaError_t e = ev ? cudaEventRecord(ev[0], st) : cudaSuccess;
    if (e == cudaSuccess)
        e = conv_layer<16, 32, EPI_HIDDEN>(c, c->X0, c->W1, c->W1c, c->p + OFF_B1, c->Z1, c->A1, nullptr, st);
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[1], st);
    if (e == cudaSuccess)
        e = conv_layer<32, 32, EPI_HIDDEN>(c, c->A1, c->W2, c->W2c, c->p + OFF_B2, c->Z2, c->A2, nullptr, st);
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[2], st);
    if (e == cudaSuccess)
        e = conv_layer<32, OUTP, EPI_OUT>(c, c->A2, c->W3, c->W3c, c->b3p, c->Y3, nullptr, nullptr, st);
    if (e == cudaSuccess && ev) e = cudaEventRecord(ev[3], st);
    return e;
}

__global__ void k_scale(float *g, int n, float s) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) g[e] *= s;
}

static cudaError_t net_forward(dns_net_ctx *c, const float *g, cudaStream_t st, cudaEvent_t *ev = nullptr) {
    const long long V = (long long)c->n * c->n * c->n;
    k_prep_input<<<nblk(V), 256, 0, st>>>(g, V, c->X0);
    if (cudaError_t e = cudaGetLastError(); e != cudaSuccess) return e;
    return net_forward_x0(c, st, ev);
}

// backward of the sample in flight (after net_forward), accumulating gradients
static cudaError_t net_backward(dns_net_ctx *c, const float *tau) {
    const long long V = (long long)c->n * c->n * c->n;
    const int lblocks = 256;
    cudaError_t e;
    k_mse<<<lblocks, 256, 0, c->stream>>>(c->Y3, tau, V, c->dY3, c->lpart);
    k_sum_d<<<1, 32, 0, c->stream>>>(c->lpart, lblocks, 1.0 / (6.0 * (double)V), c->lsum);
    const dim3 wg(c->nchunk, 27);
    // layer 3
    k_wgrad<32, OUTP><<<wg, 256, 0, c->stream>>>(c->n, c->dY3, c->A2, c->wpart, (int)((V + c->nchunk - 1) / c->nchunk));
    k_wgrad_reduce<<<nblk(27 * OUTP * 32), 256, 0, c->stream>>>(c->wpart, c->nchunk, OUTP, 32, c->gw3);
    k_colsum<<<OUTP, 256, 0, c->stream>>>(c->dY3, V, OUTP, 6, c->gb + 64);
    if ((e = conv_layer<OUTP, 32, EPI_DGRAD>(c, c->dY3, c->W3f, c->W3fc, nullptr, nullptr, c->dZ2, c->Z2,
                                             c->stream)) != cudaSuccess)
        return e;
    // layer 2
    k_wgrad<32, 32><<<wg, 256, 0, c->stream>>>(c->n, c->dZ2, c->A1, c->wpart, (int)((V + c->nchunk - 1) / c->nchunk));
    k_wgrad_reduce<<<nblk(27 * 32 * 32), 256, 0, c->stream>>>(c->wpart, c->nchunk, 32, 32, c->gw2);
    k_colsum<<<32, 256, 0, c->stream>>>(c->dZ2, V, 32, 32, c->gb + 32);
    if ((e = conv_layer<32, 32, EPI_DGRAD>(c, c->dZ2, c->W2f, c->W2fc, nullptr, nullptr, c->dZ1, c->Z1,
                                           c->stream)) != cudaSuccess)
        return e;
    // layer 1
    k_wgrad<16, 32><<<wg, 256, 0, c->stream>>>(c->n, c->dZ1, c->X0, c->wpart, (int)((V + c->nchunk - 1) / c->nchunk));
    k_wgrad_reduce<<<nblk(27 * 32 * 16), 256, 0, c->stream>>>(c->wpart, c->nchunk, 32, 16, c->gw1);
    k_colsum<<<32, 256, 0, c->stream>>>(c->dZ1, V, 32, 32, c->gb);
    return cudaGetLastError();
}

#define NK(call)                       \
    do {                               \
        cudaError_t e_ = (call);       \
        if (e_ != cudaSuccess) return DNS_ERR_CUDA; \
    } while (0)

// After the network's stream has drained: DNS_ERR_TIMEOUT if a convolution
// gave up one of its bounded waits (the status stays set).
static int net_status(dns_net_ctx *c) {
    int v = 0;
    if (cudaMemcpy(&v, c->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return DNS_ERR_CUDA;
    return v ? DNS_ERR_TIMEOUT : DNS_OK;
}

extern "C" {

int dns_net_create(int n, unsigned long long seed, void *cuda_stream, dns_net *out) {
    if (!out) return DNS_ERR_ARG;
    *out = nullptr;
    if (n < 16 || n > 256 || n % 16) return DNS_ERR_UNSUPPORTED;
    dns_net_ctx *c = new (std::nothrow) dns_net_ctx();
    if (!c) return DNS_ERR_OOM;
    c->n = n;
    const long long V = (long long)n * n * n;
    c->nchunk = (int)((V + 2047) / 2048);
    bool ok = true;
    auto al = [&](void **p, size_t b) {
        if (ok && cudaMalloc(p, b) != cudaSuccess) {
            *p = nullptr;
            ok = false;
        }
    };
    al((void **)&c->p, sizeof(float) * NET_PARAMS);
    al((void **)&c->m, sizeof(float) * NET_PARAMS);
    al((void **)&c->v, sizeof(float) * NET_PARAMS);
    al((void **)&c->gw1, sizeof(float) * 32 * 27 * 16);
    al((void **)&c->gw2, sizeof(float) * 32 * 27 * 32);
    al((void **)&c->gw3, sizeof(float) * OUTP * 27 * 32);
    al((void **)&c->gb, sizeof(float) * 72);
    al((void **)&c->W1, 2 * 32 * 27 * 16);
    al((void **)&c->W2, 2 * 32 * 27 * 32);
    al((void **)&c->W3, 2 * OUTP * 27 * 32);
    al((void **)&c->W2f, 2 * 32 * 27 * 32);
    al((void **)&c->W3f, 2 * 32 * 27 * OUTP);
    al((void **)&c->W1c, 2 * 32 * 27 * 16);
    al((void **)&c->W2c, 2 * 32 * 27 * 32);
    al((void **)&c->W3c, 2 * OUTP * 27 * 32);
    al((void **)&c->W2fc, 2 * 32 * 27 * 32);
    al((void **)&c->W3fc, 2 * 32 * 27 * OUTP);
    al((void **)&c->err, sizeof(int));
    al((void **)&c->X0, 2 * V * 16);
    al((void **)&c->A1, 2 * V * 32);
    al((void **)&c->A2, 2 * V * 32);
    al((void **)&c->dY3, 2 * V * OUTP);
    al((void **)&c->dZ2, 2 * V * 32);
    al((void **)&c->dZ1, 2 * V * 32);
    al((void **)&c->Z1, 4 * V * 32);
    al((void **)&c->Z2, 4 * V * 32);
    al((void **)&c->Y3, 4 * V * OUTP);
    al((void **)&c->b3p, sizeof(float) * OUTP);
    al((void **)&c->wpart, sizeof(float) * (size_t)c->nchunk * 27 * 32 * 32);
    al((void **)&c->lpart, sizeof(double) * 256);
    al((void **)&c->lsum, sizeof(double));
    if (ok && cudaMallocHost((void **)&c->hostd, sizeof(double) * 4) != cudaSuccess) {
        c->hostd = nullptr;
        ok = false;
    }
    if (!ok) {
        net_release(c);
        return DNS_ERR_OOM;
    }
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else if (cudaStreamCreate(&c->stream) != cudaSuccess) {
        net_release(c);
        return DNS_ERR_CUDA;
    } else {
        c->own_stream = true;
    }
    // He-style initialisation from a 64-bit LCG + Box-Muller on the host
    std::vector<float> h(NET_PARAMS, 0.f);
    unsigned long long s = seed * 6364136223846793005ULL + 1442695040888963407ULL;
    auto unif = [&]() {
        s = s * 6364136223846793005ULL + 1442695040888963407ULL;
        return ((s >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    };
    auto normal = [&]() { return std::sqrt(-2.0 * std::log(unif())) * std::cos(2.0 * M_PI * unif()); };
    for (long i = 0; i < NET_W1; ++i) h[OFF_W1 + i] = (float)(normal() * std::sqrt(2.0 / (9 * 27)));
    for (long i = 0; i < NET_W2; ++i) h[OFF_W2 + i] = (float)(normal() * std::sqrt(2.0 / (32 * 27)));
    for (long i = 0; i < NET_W3; ++i) h[OFF_W3 + i] = (float)(normal() * std::sqrt(1.0 / (32 * 27)));
    if (cudaMemcpy(c->p, h.data(), sizeof(float) * NET_PARAMS, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(c->m, 0, sizeof(float) * NET_PARAMS) != cudaSuccess ||
        cudaMemset(c->v, 0, sizeof(float) * NET_PARAMS) != cudaSuccess || net_pack(c) != cudaSuccess ||
        cudaMemset(c->err, 0, sizeof(int)) != cudaSuccess || conv_tc_attr<16, 32, EPI_HIDDEN>() != cudaSuccess ||
        conv_tc_attr<32, 32, EPI_HIDDEN>() != cudaSuccess || conv_tc_attr<32, OUTP, EPI_OUT>() != cudaSuccess ||
        conv_tc_attr<OUTP, 32, EPI_DGRAD>() != cudaSuccess || conv_tc_attr<32, 32, EPI_DGRAD>() != cudaSuccess ||
        conv_slab_attr<16, 32, EPI_HIDDEN>() != cudaSuccess || conv_slab_attr<32, 32, EPI_HIDDEN>() != cudaSuccess ||
        conv_slab_attr<32, OUTP, EPI_OUT>() != cudaSuccess || conv_slab_attr<OUTP, 32, EPI_DGRAD>() != cudaSuccess ||
        conv_slab_attr<32, 32, EPI_DGRAD>() != cudaSuccess ||
        conv_attr<16, 32, EPI_HIDDEN>() != cudaSuccess || conv_attr<32, 32, EPI_HIDDEN>() != cudaSuccess ||
        conv_attr<32, OUTP, EPI_OUT>() != cudaSuccess || conv_attr<OUTP, 32, EPI_DGRAD>() != cudaSuccess ||
        conv_attr<32, 32, EPI_DGRAD>() != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess) {
        net_release(c);
        return DNS_ERR_CUDA;
    }
    *out = c;
    return DNS_OK;
}

int dns_net_free(dns_net net) {
    if (!net) return DNS_OK;
    cudaStreamSynchronize(net->stream);
    net_release(net);
    return DNS_OK;
}

long dns_net_param_count(void) { return NET_PARAMS; }

int dns_net_set_engine(dns_net net, int engine) {
    if (!net || (engine != DNS_CONV_MMA_SYNC && engine != DNS_CONV_TCGEN05 && engine != DNS_CONV_TCGEN05_SLAB))
        return DNS_ERR_ARG;
    net->engine = engine;
    return DNS_OK;
}

int dns_net_get_engine(dns_net net, int *engine) {
    if (!net || !engine) return DNS_ERR_ARG;
    *engine = net->engine;
    return DNS_OK;
}

int dns_net_set_closure_scaling(dns_net net, double in_scale, double out_scale) {
    if (!net || !(in_scale > 0.0) || !(out_scale > 0.0) || !std::isfinite(in_scale) || !std::isfinite(out_scale))
        return DNS_ERR_ARG;
    net->in_scale = (float)in_scale;
    net->out_scale = (float)out_scale;
    return DNS_OK;
}

int dns_net_get_params(dns_net net, float *host, long count) {
    if (!net || !host || count != NET_PARAMS) return DNS_ERR_ARG;
    NK(cudaMemcpyAsync(host, net->p, sizeof(float) * NET_PARAMS, cudaMemcpyDeviceToHost, net->stream));
    NK(cudaStreamSynchronize(net->stream));
    return DNS_OK;
}

int dns_net_set_params(dns_net net, const float *host, long count) {
    if (!net || !host || count != NET_PARAMS) return DNS_ERR_ARG;
    NK(cudaMemcpyAsync(net->p, host, sizeof(float) * NET_PARAMS, cudaMemcpyHostToDevice, net->stream));
    NK(net_pack(net));
    NK(cudaStreamSynchronize(net->stream));
    return DNS_OK;
}

int dns_net_forward(dns_net net, const float *g, float *tau) {
    TraceRange trace_("dns_net_forward");
    if (!net || !g || !tau) return DNS_ERR_ARG;
    const long long V = (long long)net->n * net->n * net->n;
    NK(net_forward(net, g, net->stream));
    k_out_to_tau<<<nblk(V), 256, 0, net->stream>>>(net->Y3, V, tau, 1.0f);
    NK(cudaGetLastError());
    NK(cudaStreamSynchronize(net->stream));
    return net_status(net);
}

int dns_net_forward_profiled(dns_net net, const float *g, float *tau, int reps, double *layer_ms, double *total_ms) {
    if (!net || !g || !tau || !layer_ms || !total_ms || reps < 1 || reps > 10000) return DNS_ERR_ARG;
    const long long V = (long long)net->n * net->n * net->n;
    // per forward: [0] before it, [1..4] before layer 1 and after each layer, [5] after it
    std::vector<cudaEvent_t> ev(6 * (size_t)reps, nullptr);
    int rc = DNS_OK;
    for (auto &e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            e = nullptr;
            rc = DNS_ERR_CUDA;
            break;
        }
    for (int r = 0; r < reps && rc == DNS_OK; ++r) {
        cudaEvent_t *er = ev.data() + 6 * (size_t)r;
        if (cudaEventRecord(er[0], net->stream) != cudaSuccess || net_forward(net, g, net->stream, er + 1) != cudaSuccess)
            rc = DNS_ERR_CUDA;
        if (rc != DNS_OK) break;
        k_out_to_tau<<<nblk(V), 256, 0, net->stream>>>(net->Y3, V, tau, 1.0f);
        if (rc == DNS_OK && (cudaGetLastError() != cudaSuccess || cudaEventRecord(er[5], net->stream) != cudaSuccess))
            rc = DNS_ERR_CUDA;
    }
    if (cudaStreamSynchronize(net->stream) != cudaSuccess) rc = DNS_ERR_CUDA;
    if (rc == DNS_OK) {
        double acc[3] = {0, 0, 0};
        float ms = 0.f;
        for (int r = 0; r < reps && rc == DNS_OK; ++r) {
            const cudaEvent_t *er = ev.data() + 6 * (size_t)r;
            for (int l = 0; l < 3 && rc == DNS_OK; ++l) {
                if (cudaEventElapsedTime(&ms, er[1 + l], er[2 + l]) != cudaSuccess) rc = DNS_ERR_CUDA;
                acc[l] += ms;
            }
        }
        if (rc == DNS_OK && cudaEventElapsedTime(&ms, ev[0], ev[6 * (size_t)reps - 1]) != cudaSuccess) rc = DNS_ERR_CUDA;
        if (rc == DNS_OK) {
            for (int l = 0; l < 3; ++l) layer_ms[l] = acc[l] / reps;
            *total_ms = (double)ms / reps;
        }
    }
    for (auto &e : ev)
        if (e) cudaEventDestroy(e);
    return rc == DNS_OK ? net_status(net) : rc;
}

int dns_net_gradients(dns_net net, const float *g, const float *tau, double *loss, float *grad_host, long count) {
    TraceRange trace_("dns_net_gradients");
    if (!net || !g || !tau || (grad_host && count != NET_PARAMS)) return DNS_ERR_ARG;
    NK(cudaMemsetAsync(net->gw1, 0, sizeof(float) * 32 * 27 * 16, net->stream));
    NK(cudaMemsetAsync(net->gw2, 0, sizeof(float) * 32 * 27 * 32, net->stream));
    NK(cudaMemsetAsync(net->gw3, 0, sizeof(float) * OUTP * 27 * 32, net->stream));
    NK(cudaMemsetAsync(net->gb, 0, sizeof(float) * 72, net->stream));
    NK(cudaMemsetAsync(net->lsum, 0, sizeof(double), net->stream));
    NK(net_forward(net, g, net->stream));
    NK(net_backward(net, tau));
    if (loss) {
        NK(cudaMemcpyAsync(net->hostd, net->lsum, sizeof(double), cudaMemcpyDeviceToHost, net->stream));
    }
    if (grad_host) {
        // back to the master layout: weights [Cout][Cin][27], biases
        std::vector<float> g1(32 * 27 * 16), g2(32 * 27 * 32), g3(OUTP * 27 * 32), gb(72);
        NK(cudaMemcpyAsync(g1.data(), net->gw1, sizeof(float) * g1.size(), cudaMemcpyDeviceToHost, net->stream));
        NK(cudaMemcpyAsync(g2.data(), net->gw2, sizeof(float) * g2.size(), cudaMemcpyDeviceToHost, net->stream));
        NK(cudaMemcpyAsync(g3.data(), net->gw3, sizeof(float) * g3.size(), cudaMemcpyDeviceToHost, net->stream));
        NK(cudaMemcpyAsync(gb.data(), net->gb, sizeof(float) * gb.size(), cudaMemcpyDeviceToHost, net->stream));
        NK(cudaStreamSynchronize(net->stream));
        auto unpack = [&](const std::vector<float> &src, int cout, int cin, int cinp, float *dst) {
            for (int o = 0; o < cout; ++o)
                for (int c = 0; c < cin; ++c)
                    for (int t = 0; t < 27; ++t) dst[((long)o * cin + c) * 27 + t] = src[((long)o * 27 + t) * cinp + c];
        };
        unpack(g1, 32, 9, 16, grad_host + OFF_W1);
        unpack(g2, 32, 32, 32, grad_host + OFF_W2);
        unpack(g3, 6, 32, 32, grad_host + OFF_W3);
        std::memcpy(grad_host + OFF_B1, gb.data(), sizeof(float) * 32);
        std::memcpy(grad_host + OFF_B2, gb.data() + 32, sizeof(float) * 32);
        std::memcpy(grad_host + OFF_B3, gb.data() + 64, sizeof(float) * 6);
    }
    NK(cudaStreamSynchronize(net->stream));
    if (loss) *loss = net->hostd[0];
    return net_status(net);
}

int dns_net_train_step(dns_net net, int nsamples, const float *g, const float *tau, double lr, double *loss) {
    TraceRange trace_("dns_net_train_step");
    if (!net || !g || !tau || nsamples < 1 || !(lr > 0.0)) return DNS_ERR_ARG;
    const long long V = (long long)net->n * net->n * net->n;
    NK(cudaMemsetAsync(net->gw1, 0, sizeof(float) * 32 * 27 * 16, net->stream));
    NK(cudaMemsetAsync(net->gw2, 0, sizeof(float) * 32 * 27 * 32, net->stream));
    NK(cudaMemsetAsync(net->gw3, 0, sizeof(float) * OUTP * 27 * 32, net->stream));
    NK(cudaMemsetAsync(net->gb, 0, sizeof(float) * 72, net->stream));
    NK(cudaMemsetAsync(net->lsum, 0, sizeof(double), net->stream));
    for (int i = 0; i < nsamples; ++i) {
        NK(net_forward(net, g + (long long)i * 9 * V, net->stream));
        NK(net_backward(net, tau + (long long)i * 6 * V));
    }
    // Adam on the minibatch-mean gradient
    net->step += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - std::pow(b1, (float)net->step), c2 = 1.f - std::pow(b2, (float)net->step);
    const float inv = 1.f / (float)nsamples;
    struct Blk {
        float *g;
        int n;
    } grads[4] = {{net->gw1, 32 * 27 * 16}, {net->gw2, 32 * 27 * 32}, {net->gw3, OUTP * 27 * 32}, {net->gb, 72}};
    for (auto &b : grads) k_scale<<<nblk(b.n), 256, 0, net->stream>>>(b.g, b.n, inv);
    const float lrf = (float)lr;
    k_adam<<<nblk(NET_W1), 256, 0, net->stream>>>(net->p + OFF_W1, net->m + OFF_W1, net->v + OFF_W1, net->gw1,
                                                   (int)NET_W1, 1, 32, 9, 16, lrf, b1, b2, eps, c1, c2);
    k_adam<<<1, 256, 0, net->stream>>>(net->p + OFF_B1, net->m + OFF_B1, net->v + OFF_B1, net->gb, 32, 0, 0, 0, 0,
                                       lrf, b1, b2, eps, c1, c2);
    k_adam<<<nblk(NET_W2), 256, 0, net->stream>>>(net->p + OFF_W2, net->m + OFF_W2, net->v + OFF_W2, net->gw2,
                                                   (int)NET_W2, 1, 32, 32, 32, lrf, b1, b2, eps, c1, c2);
    k_adam<<<1, 256, 0, net->stream>>>(net->p + OFF_B2, net->m + OFF_B2, net->v + OFF_B2, net->gb + 32, 32, 0, 0, 0,
                                       0, lrf, b1, b2, eps, c1, c2);
    k_adam<<<nblk(NET_W3), 256, 0, net->stream>>>(net->p + OFF_W3, net->m + OFF_W3, net->v + OFF_W3, net->gw3,
                                                   (int)NET_W3, 1, 6, 32, 32, lrf, b1, b2, eps, c1, c2);
    k_adam<<<1, 256, 0, net->stream>>>(net->p + OFF_B3, net->m + OFF_B3, net->v + OFF_B3, net->gb + 64, 6, 0, 0, 0,
                                       0, lrf, b1, b2, eps, c1, c2);
    NK(cudaGetLastError());
    NK(net_pack(net));
    if (loss) NK(cudaMemcpyAsync(net->hostd, net->lsum, sizeof(double), cudaMemcpyDeviceToHost, net->stream));
    NK(cudaStreamSynchronize(net->stream));
    if (loss) *loss = net->hostd[0] / nsamples;
    (void)V;
    return net_status(net);
}

}  // extern "C"

// ---------------------------------------------------------------- closure and training data
static float2 *make_twiddles_f(int N) {
    std::vector<float2> h(N);
    for (int m = 0; m < N; ++m) {
        const double a = 2.0 * M_PI * m / N;
        h[m] = make_float2((float)std::cos(a), (float)-std::sin(a));
    }
    float2 *d = nullptr;
    if (cudaMalloc(&d, sizeof(float2) * N) != cudaSuccess) return nullptr;
    if (cudaMemcpy(d, h.data(), sizeof(float2) * N, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(d);
        return nullptr;
    }
    return d;
}

namespace dns {
struct LesClosure {
    dns_net_ctx *net = nullptr;  // not owned; null selects the Smagorinsky stresses
    float smag_c2 = 0.f;         // (C_s Delta)^2 of the Smagorinsky model
    int n = 0;
    float2 *tw = nullptr, *gc = nullptr, *thc = nullptr;
    float *gr = nullptr, *tau = nullptr;
};

void les_closure_release(LesClosure *c) {
    if (!c) return;
    void *b[] = {c->tw, c->gc, c->thc, c->gr, c->tau};
    for (void *p : b)
        if (p) cudaFree(p);
    delete c;
}

cudaError_t les_closure_forcing(LesClosure *c, const Geo &g, const void *U, void *Fext, cudaStream_t st) {
    const int n = c->n;
    const long long V = (long long)n * n * n;
    cudaError_t e;
    k_compact_to_full_c<<<nblk(9 * V), 256, 0, st>>>(g, (const float2 *)U, c->gc, 1, 1.0f / (float)V);
    if ((e = c2c(n, c->gc, c->tw, 9, +1, st)) != cudaSuccess) return e;
    if (c->net) {
        k_real_part<<<nblk(9 * V), 256, 0, st>>>(c->gc, 9 * V, c->gr, c->net->in_scale);
        if ((e = net_forward(c->net, c->gr, st)) != cudaSuccess) return e;
        k_out_to_tau<<<nblk(V), 256, 0, st>>>(c->net->Y3, V, c->tau, c->net->out_scale);
    } else {
        k_real_part<<<nblk(9 * V), 256, 0, st>>>(c->gc, 9 * V, c->gr, 1.0f);
        k_smagorinsky<<<nblk(V), 256, 0, st>>>(c->gr, V, c->smag_c2, c->tau);
    }
    k_real_to_c<<<nblk(6 * V), 256, 0, st>>>(c->tau, 6 * V, c->thc);
    if ((e = c2c(n, c->thc, c->tw, 6, -1, st)) != cudaSuccess) return e;
    k_closure_forcing<<<nblk(g.sS), 256, 0, st>>>(g, c->thc, (float2 *)Fext);
    return cudaGetLastError();
}
}  // namespace dns

// compact N-mesh state -> full half-spectrum layout on the n mesh, |k_i| <= kc, times scale
__global__ void k_filter_to_half(dns::Geo g, const float2 *__restrict__ U, int n, int kc, float scale,
                                 float2 *__restrict__ out) {
    const int nh = n / 2 + 1;
    const long long total = 3LL * n * n * nh;
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int kz = (int)(e % nh);
    const long long r = e / nh;
    const int iy = (int)(r % n), ix = (int)((r / n) % n), c = (int)(r / ((long long)n * n));
    const int kx = fft_k(ix, n), ky = fft_k(iy, n);
    float2 v = make_float2(0.f, 0.f);
    if (abs(kx) <= kc && abs(ky) <= kc && kz <= kc && abs(kx) <= g.K && abs(ky) <= g.K && kz <= g.K) {
        const int cx = kx >= 0 ? kx : kx + g.Kx, cy = ky >= 0 ? ky : ky + g.Kx;
        const float2 u = U[c * g.sS + ((long long)cx * g.Kx + cy) * g.Kzp + kz];
        v = make_float2(u.x * scale, u.y * scale);
    }
    out[e] = v;
}

struct dns_les_builder_ctx {
    int N = 0, n = 0;
    float2 *twN = nullptr, *twn = nullptr, *bigc = nullptr, *smallc = nullptr, *ubc = nullptr;
};

static void builder_release(dns_les_builder_ctx *b) {
    if (!b) return;
    void *p[] = {b->twN, b->twn, b->bigc, b->smallc, b->ubc};
    for (void *q : p)
        if (q) cudaFree(q);
    delete b;
}

extern "C" {

int dns_les_builder_create(int N, int n, dns_les_builder *out) {
    if (!out) return DNS_ERR_ARG;
    *out = nullptr;
    if (!c2c_supported(N) || !c2c_supported(n) || n > N) return DNS_ERR_UNSUPPORTED;
    dns_les_builder_ctx *b = new (std::nothrow) dns_les_builder_ctx();
    if (!b) return DNS_ERR_OOM;
    b->N = N;
    b->n = n;
    const long long VN = (long long)N * N * N, Vn = (long long)n * n * n;
    b->twN = make_twiddles_f(N);
    b->twn = make_twiddles_f(n);
    bool ok = b->twN && b->twn;
    if (ok && cudaMalloc(&b->bigc, sizeof(float2) * 9 * VN) != cudaSuccess) { b->bigc = nullptr; ok = false; }
    if (ok && cudaMalloc(&b->smallc, sizeof(float2) * 9 * Vn) != cudaSuccess) { b->smallc = nullptr; ok = false; }
    if (ok && cudaMalloc(&b->ubc, sizeof(float2) * 3 * Vn) != cudaSuccess) { b->ubc = nullptr; ok = false; }
    if (!ok) {
        builder_release(b);
        return DNS_ERR_OOM;
    }
    *out = b;
    return DNS_OK;
}

int dns_les_builder_free(dns_les_builder b) {
    if (b) {
        cudaDeviceSynchronize();
        builder_release(b);
    }
    return DNS_OK;
}

int dns_les_builder_run(dns_les_builder b, dns_handle dns, float *g, float *tau, void *ubar_hat) {
    TraceRange trace_("dns_les_builder_run");
    if (!b || !dns || !g || !tau) return DNS_ERR_ARG;
    dns::InternalView v;
    if (dns::internal_view(dns, &v) || v.N != b->N) return DNS_ERR_ARG;
    if (v.dtype != DNS_F32) return DNS_ERR_UNSUPPORTED;
    const int N = b->N, n = b->n, kc = (n - 1) / 3;
    const long long VN = (long long)N * N * N, Vn = (long long)n * n * n;
    cudaStream_t st = v.stream;
    const float2 *U = (const float2 *)v.U0;
    const float invN3 = 1.0f / (float)VN;
    // u on the DNS mesh, its six products, forward
    k_compact_to_full_c<<<nblk(3 * VN), 256, 0, st>>>(v.g, U, b->bigc, 0, invN3);
    NK(c2c(N, b->bigc, b->twN, 3, +1, st));
    k_products<<<nblk(6 * VN), 256, 0, st>>>(b->bigc, VN, b->bigc + 3 * VN);
    NK(c2c(N, b->bigc + 3 * VN, b->twN, 6, -1, st));
    // filt(u_i u_j) at the LES points: cutoff, move to the n mesh, inverse (1/N^3 folded in)
    k_filter_full<<<nblk(6 * Vn), 256, 0, st>>>(b->bigc + 3 * VN, N, b->smallc, n, 6, kc, invN3);
    NK(c2c(n, b->smallc, b->twn, 6, +1, st));
    // ubar at the LES points
    k_compact_to_full_c<<<nblk(3 * VN), 256, 0, st>>>(v.g, U, b->bigc, 0, 1.0f);
    k_filter_full<<<nblk(3 * Vn), 256, 0, st>>>(b->bigc, N, b->ubc, n, 3, kc, invN3);
    NK(c2c(n, b->ubc, b->twn, 3, +1, st));
    k_tau_from_parts<<<nblk(6 * Vn), 256, 0, st>>>(b->smallc, b->ubc, Vn, tau);
    // gradients d_j ubar_i
    k_compact_to_full_c<<<nblk(9 * VN), 256, 0, st>>>(v.g, U, b->bigc, 1, 1.0f);
    k_filter_full<<<nblk(9 * Vn), 256, 0, st>>>(b->bigc, N, b->smallc, n, 9, kc, invN3);
    NK(c2c(n, b->smallc, b->twn, 9, +1, st));
    k_real_part<<<nblk(9 * Vn), 256, 0, st>>>(b->smallc, 9 * Vn, g, 1.0f);
    if (ubar_hat) {
        const float scale = (float)((double)Vn / (double)VN);
        k_filter_to_half<<<nblk(3LL * n * n * (n / 2 + 1)), 256, 0, st>>>(v.g, U, n, kc, scale, (float2 *)ubar_hat);
    }
    NK(cudaGetLastError());
    NK(cudaStreamSynchronize(st));
    return DNS_OK;
}

// Buffers of a closure on the N^3 mesh of handle view v (net or Smagorinsky).
static int closure_attach(dns_handle h, const dns::InternalView &v, dns_net net, float smag_c2) {
    dns::LesClosure *c = new (std::nothrow) dns::LesClosure();
    if (!c) return DNS_ERR_OOM;
    c->net = net;
    c->smag_c2 = smag_c2;
    c->n = v.N;
    const long long V = (long long)v.N * v.N * v.N;
    c->tw = make_twiddles_f(v.N);
    bool ok = c->tw != nullptr;
    if (ok && cudaMalloc(&c->gc, sizeof(float2) * 9 * V) != cudaSuccess) { c->gc = nullptr; ok = false; }
    if (ok && cudaMalloc(&c->thc, sizeof(float2) * 6 * V) != cudaSuccess) { c->thc = nullptr; ok = false; }
    if (ok && cudaMalloc(&c->gr, sizeof(float) * 9 * V) != cudaSuccess) { c->gr = nullptr; ok = false; }
    if (ok && cudaMalloc(&c->tau, sizeof(float) * 6 * V) != cudaSuccess) { c->tau = nullptr; ok = false; }
    if (!ok) {
        dns::les_closure_release(c);
        return DNS_ERR_OOM;
    }
    return dns::internal_set_closure(h, c);
}

int dns_les_set_closure(dns_handle h, dns_net net) {
    if (!h) return DNS_ERR_ARG;
    if (!net) return dns::internal_set_closure(h, nullptr);
    dns::InternalView v;
    if (dns::internal_view(h, &v)) return DNS_ERR_ARG;
    if (v.dtype != DNS_F32 || v.N != net->n || !c2c_supported(v.N) || v.g.nb != 1) return DNS_ERR_UNSUPPORTED;
    return closure_attach(h, v, net, 0.f);
}

int dns_les_set_smagorinsky(dns_handle h, double cs, double delta) {
    if (!h || !(cs >= 0.0) || !std::isfinite(cs) || !std::isfinite(delta)) return DNS_ERR_ARG;
    dns::InternalView v;
    if (dns::internal_view(h, &v)) return DNS_ERR_ARG;
    if (v.dtype != DNS_F32 || !c2c_supported(v.N) || v.g.nb != 1) return DNS_ERR_UNSUPPORTED;
    const double d = delta > 0.0 ? delta : 2.0 * M_PI / v.N;
    return closure_attach(h, v, nullptr, (float)(cs * cs * d * d));
}

}  // extern "C"
