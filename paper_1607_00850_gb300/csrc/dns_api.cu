// C-ABI of the single-GPU pseudo-spectral solver (include/dns.h).
//
// One RK4 step = 4 stages x 6 passes (dns_passes.cuh).  The step is captured
// once into a CUDA graph and replayed.  All buffers are allocated at
// dns_init; nothing is allocated on the stepping path.
#include "dns.h"
#include "dns_internal.h"
#include "dns_passes.cuh"

#include <cmath>
#include <cstdio>
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
#define DNS_SIZES(X)                                                                                            \
    X(6) X(8) X(12) X(16) X(18) X(24) X(32) X(36) X(48) X(54) X(64) X(72) X(96) X(108) X(128) X(144) X(162) X(192) \
        X(216) X(256) X(288) X(324) X(384) X(432) X(486) X(512) X(576) X(648) X(768) X(864) X(972) X(1024)
#define DNS_DECL(n) bool get_passes_##n(int, PassSet *);
DNS_SIZES(DNS_DECL)
#undef DNS_DECL

static PassGetter getter_for(int N) {
    switch (N) {
#define DNS_CASE(n) \
    case n:         \
        return get_passes_##n;
        DNS_SIZES(DNS_CASE)
#undef DNS_CASE
        default:
            return nullptr;
    }
}
}  // namespace dns

using dns::Geo;

// Every device buffer of a handle sits between two guard regions of
// kGuardBytes filled with kGuardByte; dns_check_guards reads them back, so a
// kernel that writes past either end of a buffer is caught.
constexpr size_t kGuardBytes = 256;  // keeps the buffer itself 256-byte aligned
constexpr unsigned char kGuardByte = 0xA5;
struct GuardedAlloc {
    void *base, *user;
    size_t bytes;
};

struct dns_ctx {
    int N = 0, dtype = 0;
    double nu = 0, dt = 0, t = 0;
    long step = 0;
    Geo g{};
    dns::PassSet ps{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool same_type = false;   // field and accumulator types coincide
    size_t creal = 0, cacc = 0, cio = 0;  // bytes per complex element
    void *U = nullptr, *U0 = nullptr, *U1 = nullptr, *A = nullptr, *B = nullptr;
    void *io = nullptr, *rin = nullptr, *rout = nullptr, *tw = nullptr;
    void *Om = nullptr, *rom = nullptr;  // curl of the stage input (state boxes / rhs input)
    double *partials = nullptr, *sums = nullptr, *Ek = nullptr;
    double *nu_box = nullptr;  // per-box viscosity when several boxes share the context
    int *err = nullptr;        // device status word: [0] code, [1] source line, [2..3] address (Geo::err)
    unsigned long long *rng = nullptr;  // device table of the address ranges kernels may touch (checked builds)
    int nblk = 0, smax = 0;
    double *host = nullptr;  // pinned read-back area
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long bytes = 0;
    std::vector<GuardedAlloc> allocs;  // every device buffer, with its guard regions
    int plan[5] = {0, 0, 0, 0, 0};  // variant of P1, P2, P3, P4, P5a
    int integrator = 0;             // DNS_RK4 or DNS_IFRK4
    dns::LesClosure *closure = nullptr;  // learned subgrid closure (LES handles), or nullptr
    void *Fext = nullptr;                // its forcing on the stored modes
    int closure_every_stage = 1;         // 0: evaluated from the step's first stage input only
    // asynchronous host I/O (created on first use): a copy-in and a copy-out
    // stream, one staging buffer in and two out (full spectral layout)
    cudaStream_t s_in = nullptr, s_out = nullptr;
    void *io_in = nullptr, *io_out[2] = {nullptr, nullptr};
    cudaEvent_t in_copied = nullptr, in_free = nullptr, out_ready[2] = {nullptr, nullptr},
                out_copied[2] = {nullptr, nullptr};
    int out_slot = 0;
};

static thread_local cudaError_t g_last_cuda = cudaSuccess;

#define CK(call)                              \
    do {                                      \
        cudaError_t e_ = (call);              \
        if (e_ != cudaSuccess) {              \
            g_last_cuda = e_;                 \
            return DNS_ERR_CUDA;              \
        }                                     \
    } while (0)

#define DNS_NPASS 6

static const double RK_A[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
static const double RK_B[3] = {0.5, 0.5, 1.0};

static void drop_async_io(dns_ctx *h);

// Index-checked builds: the device table of address ranges (its layout in
// dns_check.cuh) lists every device buffer of the handle without its guard
// regions, plus up to two caller buffers of the call in progress.  Rewritten
// (synchronously) whenever a buffer is allocated or freed and around calls
// that hand the kernels a caller's device buffer.  A no-op otherwise.
static void refresh_ranges(dns_ctx *h, const void *p1 = nullptr, size_t b1 = 0, const void *p2 = nullptr,
                           size_t b2 = 0) {
#ifdef DNS_CHECKED
    if (!h->rng) return;
    std::vector<unsigned long long> t(1, 0ull);
    auto add = [&](const void *p, size_t b) {
        if (!p || !b || t[0] >= (unsigned long long)dns::kMaxCheckRanges) return;
        t.push_back((unsigned long long)p);
        t.push_back((unsigned long long)p + b);
        ++t[0];
    };
    for (const GuardedAlloc &a : h->allocs) add(a.user, a.bytes);
    add(p1, b1);
    add(p2, b2);
    cudaMemcpy(h->rng, t.data(), t.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice);
#else
    (void)h;
    (void)p1;
    (void)b1;
    (void)p2;
    (void)b2;
#endif
}

static void release(dns_ctx *h) {
    if (!h) return;
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    if (h->host) cudaFreeHost(h->host);
    if (h->closure) dns::les_closure_release(h->closure);
    drop_async_io(h);
    for (const GuardedAlloc &a : h->allocs) cudaFree(a.base);
    h->allocs.clear();
    if (h->rng) cudaFree(h->rng);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

static int dev_alloc(dns_ctx *h, void **p, size_t bytes) {
    void *base = nullptr;
    *p = nullptr;
    if (cudaMalloc(&base, bytes + 2 * kGuardBytes) != cudaSuccess) {
        cudaGetLastError();
        return DNS_ERR_OOM;
    }
    char *user = static_cast<char *>(base) + kGuardBytes;
    cudaError_t e = cudaMemset(base, kGuardByte, kGuardBytes);
    if (e == cudaSuccess) e = cudaMemset(user + bytes, kGuardByte, kGuardBytes);
    if (e != cudaSuccess) {
        g_last_cuda = e;
        cudaFree(base);
        return DNS_ERR_CUDA;
    }
    h->allocs.push_back({base, user, bytes});
    h->bytes += (long long)bytes;
    *p = user;
    refresh_ranges(h);
    return DNS_OK;
}

static void dev_free(dns_ctx *h, void *p) {
    for (size_t i = 0; i < h->allocs.size(); ++i)
        if (h->allocs[i].user == p) {
            cudaFree(h->allocs[i].base);
            h->bytes -= (long long)h->allocs[i].bytes;
            h->allocs.erase(h->allocs.begin() + (long)i);
            refresh_ranges(h);
            return;
        }
}

// DNS_OK if every guard region of every buffer still holds kGuardByte,
// DNS_ERR_GUARD if one was overwritten (call after the work has drained).
static int check_guards(dns_ctx *h) {
    std::vector<unsigned char> buf(kGuardBytes);
    for (const GuardedAlloc &a : h->allocs)
        for (int side = 0; side < 2; ++side) {
            const char *src = side == 0 ? static_cast<const char *>(a.base) : static_cast<const char *>(a.user) + a.bytes;
            cudaError_t e = cudaMemcpy(buf.data(), src, kGuardBytes, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) {
                g_last_cuda = e;
                return DNS_ERR_CUDA;
            }
            for (unsigned char b : buf)
                if (b != kGuardByte) return DNS_ERR_GUARD;
        }
    return DNS_OK;
}

static inline int grid_for(long long total) {
    long long b = (total + 255) / 256;
    return (int)(b < 4864 ? (b < 1 ? 1 : b) : 4864);
}

// --------------------------------------------------------------- conversions
static inline unsigned row_threads(int n) {
    const int t = (n + 31) / 32 * 32;
    return (unsigned)(t < 1024 ? t : 1024);
}
// full -> compact (cmp2: a second compact copy, or nullptr)
template <typename Tin, typename Tout, typename Tout2>
static cudaError_t to_compact(const dns_ctx *h, const void *full, void *cmp, void *cmp2) {
    const dim3 grid((unsigned)h->g.Kx, (unsigned)h->g.Kx, 3);
    dns::k_full_to_compact<Tin, Tout, Tout2><<<grid, row_threads(h->g.Kz), 0, h->stream>>>(
        h->g, (const Tin *)full, (Tout *)cmp, (Tout2 *)cmp2);
    return cudaGetLastError();
}
template <typename Tin, typename Tout>
static cudaError_t to_full(const dns_ctx *h, const void *cmp, void *full) {
    const dim3 grid((unsigned)h->N, (unsigned)h->N, 3);
    dns::k_compact_to_full<Tin, Tout><<<grid, row_threads(h->N / 2 + 1), 0, h->stream>>>(h->g, (const Tin *)cmp,
                                                                                         (Tout *)full);
    return cudaGetLastError();
}

// elementwise copy between compact buffers of different complex types
template <typename Tin, typename Tout>
__global__ void k_convert(const Tin *__restrict__ a, Tout *__restrict__ b, long long n, dns::Chk ck) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const Tin v = DNS_LD(ck, a + e);
        Tout o;
        o.x = v.x;
        o.y = v.y;
        DNS_ST(ck, b + e, o);
    }
}

// full (io type) -> compact (real type) and compact (acc type)
static cudaError_t full_to_state(dns_ctx *h, const void *full, void *dst_real, void *dst_acc) {
    // one pass over the input writes both copies (dst_real is never nullptr)
    if (h->dtype == DNS_F32) return to_compact<float2, float2, float2>(h, full, dst_real, dst_acc);
    if (h->dtype == DNS_F64) return to_compact<double2, double2, double2>(h, full, dst_real, dst_acc);
    return to_compact<double2, float2, double2>(h, full, dst_real, dst_acc);
}

// compact (acc type) -> full (io type); io type == acc type in every mode
static cudaError_t acc_to_full(dns_ctx *h, const void *cmp, void *full) {
    if (h->dtype == DNS_F32) return to_full<float2, float2>(h, cmp, full);
    return to_full<double2, double2>(h, cmp, full);
}

// --------------------------------------------------------------- the path
static cudaError_t launch_front(dns_ctx *h, const void *Uin, const void *Omin) {
    cudaError_t e;
    const double scale = 1.0 / ((double)h->N * h->N * h->N);
    if ((e = h->ps.p1[h->plan[0]](h->g, h->tw, Uin, Omin, h->A, scale, h->stream)) != cudaSuccess) return e;
    if ((e = h->ps.p2[h->plan[1]](h->g, h->tw, h->A, h->B, h->stream)) != cudaSuccess) return e;
    if ((e = h->ps.p3[h->plan[2]](h->g, h->tw, h->B, h->stream)) != cudaSuccess) return e;
    return h->ps.p4[h->plan[3]](h->g, h->tw, h->B, h->A, h->stream);
}

static dns::UpdateArgsErased stage_args(const dns_ctx *h, int s) {
    dns::UpdateArgsErased a{};
    a.U = (s == 0 && h->same_type) ? h->U0 : h->U;
    a.U0 = h->U0;
    a.U1 = h->U1;
    a.Uout = (s < 3 || !h->same_type) ? h->U : nullptr;
    a.U0out = (s == 3) ? h->U0 : nullptr;
    a.dU = nullptr;
    a.Om = h->Om;
    a.Fext = h->closure ? h->Fext : nullptr;
    a.nu = h->nu;
    a.nu_box = h->nu_box;
    a.adt = RK_A[s] * h->dt;
    a.bdt = s < 3 ? RK_B[s] * h->dt : 0.0;
    a.dt = h->dt;
    a.stage = s;
    a.ifrk = h->integrator == DNS_IFRK4;
    return a;
}

// The back end of a stage: forward x transform and update, either as P5a +
// P5b or fused (plan[4] >= NCOLV); `mark` runs after each of the two slots
// (after the fused launch and again with nothing in between).
template <class Mark>
static cudaError_t launch_back(dns_ctx *h, const Geo &g, const dns::UpdateArgsErased &a, const Mark &mark) {
    cudaError_t e;
    const int v = h->plan[4];
    if (v >= dns::PassSet::NCOLV) {
        if ((e = h->ps.p5f[v - dns::PassSet::NCOLV](g, h->tw, h->A, a, h->stream)) != cudaSuccess) return e;
        if ((e = mark()) != cudaSuccess) return e;
        return mark();
    }
    if ((e = h->ps.p5a[v](g, h->tw, h->A, h->B, h->stream)) != cudaSuccess) return e;
    if ((e = mark()) != cudaSuccess) return e;
    if ((e = h->ps.p5b(g, h->B, a, h->stream)) != cudaSuccess) return e;
    return mark();
}

static cudaError_t no_mark() { return cudaSuccess; }

// Enqueue one RK4 step; if ev != nullptr record ev[1 + i] after launch i.
static cudaError_t enqueue_step(dns_ctx *h, cudaEvent_t *ev) {
    cudaError_t e;
    int li = 0;
    auto mark = [&]() -> cudaError_t {
        if (!ev) return cudaSuccess;
        return cudaEventRecord(ev[++li], h->stream);
    };
    const double scale = 1.0 / ((double)h->N * h->N * h->N);
    for (int s = 0; s < 4; ++s) {
        dns::UpdateArgsErased a = stage_args(h, s);
        if (h->closure && (s == 0 || h->closure_every_stage)) {  // subgrid forcing from this stage's input
            if ((e = dns::les_closure_forcing(h->closure, h->g, a.U, h->Fext, h->stream)) != cudaSuccess) return e;
        }
        if ((e = h->ps.p1[h->plan[0]](h->g, h->tw, a.U, h->Om, h->A, scale, h->stream)) != cudaSuccess) return e;
        if ((e = mark()) != cudaSuccess) return e;
        if ((e = h->ps.p2[h->plan[1]](h->g, h->tw, h->A, h->B, h->stream)) != cudaSuccess) return e;
        if ((e = mark()) != cudaSuccess) return e;
        if ((e = h->ps.p3[h->plan[2]](h->g, h->tw, h->B, h->stream)) != cudaSuccess) return e;
        if ((e = mark()) != cudaSuccess) return e;
        if ((e = h->ps.p4[h->plan[3]](h->g, h->tw, h->B, h->A, h->stream)) != cudaSuccess) return e;
        if ((e = mark()) != cudaSuccess) return e;
        if ((e = launch_back(h, h->g, a, mark)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// --------------------------------------------------------------- per-box state I/O
static inline void *box_ptr(void *base, long long elems, size_t eb, int b) {
    return (char *)base + (size_t)b * (size_t)elems * eb;
}

// omega^ of box b's stage input (the next P1 reads it)
static cudaError_t curl_box(dns_ctx *h, int b) {
    Geo g1 = h->g;
    g1.nb = 1;
    return h->ps.curl(g1, box_ptr(h->U, h->g.bS, h->creal, b), box_ptr(h->Om, h->g.bS, h->creal, b), h->stream);
}

// full-layout field (host or device) -> box b's stage input and step-start state
static int set_state(dns_ctx *h, int b, const void *uhat, int on_device) {
    const size_t bytes = 3ull * h->N * h->N * (h->N / 2 + 1) * h->cio;
    const void *src = uhat;
    if (!on_device) {
        CK(cudaMemcpyAsync(h->io, uhat, bytes, cudaMemcpyHostToDevice, h->stream));
        src = h->io;
    } else {
        refresh_ranges(h, uhat, bytes);
    }
    CK(full_to_state(h, src, box_ptr(h->U, h->g.bS, h->creal, b), box_ptr(h->U0, h->g.bS, h->cacc, b)));
    CK(curl_box(h, b));
    CK(cudaStreamSynchronize(h->stream));
    if (on_device) refresh_ranges(h);
    return DNS_OK;
}

static int get_state(dns_ctx *h, int b, void *uhat, int on_device) {
    const size_t bytes = 3ull * h->N * h->N * (h->N / 2 + 1) * h->cio;
    const void *u0 = box_ptr(h->U0, h->g.bS, h->cacc, b);
    if (on_device) {
        refresh_ranges(h, uhat, bytes);
        CK(acc_to_full(h, u0, uhat));
    } else {
        CK(acc_to_full(h, u0, h->io));
        CK(cudaMemcpyAsync(uhat, h->io, bytes, cudaMemcpyDeviceToHost, h->stream));
    }
    CK(cudaStreamSynchronize(h->stream));
    if (on_device) refresh_ranges(h);
    return DNS_OK;
}

static int stats_sums_box(dns_ctx *h, int b, double *se, double *sd) {
    const void *u0 = box_ptr(h->U0, h->g.bS, h->cacc, b);
    if (h->dtype == DNS_F32)
        dns::k_energy_partials<float><<<h->nblk, 256, 0, h->stream>>>(h->g, (const float2 *)u0, h->partials);
    else
        dns::k_energy_partials<double><<<h->nblk, 256, 0, h->stream>>>(h->g, (const double2 *)u0, h->partials);
    CK(cudaGetLastError());
    dns::k_sum_partials<<<1, 32, 0, h->stream>>>(h->partials, h->nblk, 2, h->sums);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(h->host, h->sums, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    *se = h->host[0];
    *sd = h->host[1];
    return DNS_OK;
}

// --------------------------------------------------------------- handles
// One context holds nb boxes of one mesh size: every pass covers all of
// them in one launch.  nu_host[b] is box b's viscosity.
static int ctx_create(int N, int nb, const double *nu_host, double dt, int dtype, cudaStream_t stream,
                      dns_ctx **out) {
    if (dtype < DNS_F32 || dtype > DNS_F32_ACC64 || nb < 1 || !nu_host) return DNS_ERR_ARG;
    if (!(dt > 0.0) || !std::isfinite(dt)) return DNS_ERR_ARG;
    for (int b = 0; b < nb; ++b)
        if (!(nu_host[b] > 0.0) || !std::isfinite(nu_host[b])) return DNS_ERR_ARG;
    dns::PassGetter get = dns::getter_for(N);
    if (!get) return DNS_ERR_UNSUPPORTED;
    dns_ctx *h = new (std::nothrow) dns_ctx();
    if (!h) return DNS_ERR_OOM;
    h->N = N;
    h->dtype = dtype;
    h->nu = nu_host[0];
    h->dt = dt;
    if (!get(dtype, &h->ps)) {
        delete h;
        return DNS_ERR_UNSUPPORTED;
    }
#ifdef DNS_CHECKED
    // the address-range table, filled by every dev_alloc below
    if (cudaMalloc((void **)&h->rng, sizeof(unsigned long long) * (1 + 2 * dns::kMaxCheckRanges)) != cudaSuccess ||
        cudaMemset(h->rng, 0, sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        if (h->rng) cudaFree(h->rng);
        delete h;
        return DNS_ERR_OOM;
    }
#endif
    const int K = (N - 1) / 3;
    Geo &g = h->g;
    g.N = N;
    g.K = K;
    g.Kx = 2 * K + 1;
    g.Kz = K + 1;
    g.Kzp = (g.Kz + 3) / 4 * 4;
    g.sS = (long long)g.Kx * g.Kx * g.Kzp;
    g.sA = (long long)N * g.Kx * g.Kzp;
    g.sB = (long long)N * N * g.Kzp;
    g.nb = nb;
    g.bS = 3 * g.sS;
    g.bA = 6 * g.sA;
    g.bB = 6 * g.sB;
    h->creal = dtype == DNS_F64 ? 16 : 8;
    h->cacc = dtype == DNS_F32 ? 8 : 16;
    h->cio = h->cacc;
    h->same_type = h->creal == h->cacc;
    int rc = DNS_OK;
    const size_t nfull = 3ull * N * N * (N / 2 + 1);
    h->nblk = 2 * 152;
    h->smax = (int)std::floor(std::sqrt(3.0) * K + 0.5) + 1;
    if (!rc) rc = dev_alloc(h, &h->U, nb * 3 * g.sS * h->creal);
    if (!rc) rc = dev_alloc(h, &h->U0, nb * 3 * g.sS * h->cacc);
    if (!rc) rc = dev_alloc(h, &h->U1, nb * 3 * g.sS * h->cacc);
    if (!rc) rc = dev_alloc(h, &h->A, nb * 6 * g.sA * h->creal);
    if (!rc) rc = dev_alloc(h, &h->B, nb * 6 * g.sB * h->creal);
    if (!rc) rc = dev_alloc(h, &h->io, nfull * h->cio);
    if (!rc) rc = dev_alloc(h, &h->rin, 3 * g.sS * h->creal);
    if (!rc) rc = dev_alloc(h, &h->Om, nb * 3 * g.sS * h->creal);
    if (!rc) rc = dev_alloc(h, &h->rom, 3 * g.sS * h->creal);
    if (!rc) rc = dev_alloc(h, &h->rout, 3 * g.sS * h->cacc);
    if (!rc) rc = dev_alloc(h, &h->tw, (size_t)N * h->creal);
    if (!rc) rc = dev_alloc(h, (void **)&h->partials, sizeof(double) * 2 * h->nblk);
    if (!rc) rc = dev_alloc(h, (void **)&h->sums, sizeof(double) * 2);
    if (!rc) rc = dev_alloc(h, (void **)&h->Ek, sizeof(double) * h->smax);
    if (!rc && nb > 1) rc = dev_alloc(h, (void **)&h->nu_box, sizeof(double) * nb);
    if (!rc) rc = dev_alloc(h, (void **)&h->err, 4 * sizeof(int));
    g.err = h->err;
    g.rng = h->rng;
    if (!rc && cudaMallocHost((void **)&h->host, sizeof(double) * (4 + h->smax)) != cudaSuccess) {
        h->host = nullptr;
        rc = DNS_ERR_OOM;
    }
    if (rc) {
        release(h);
        return rc;
    }
    if (stream) {
        h->stream = stream;
    } else {
        if (cudaStreamCreate(&h->stream) != cudaSuccess) {
            h->stream = nullptr;
            release(h);
            return DNS_ERR_CUDA;
        }
        h->own_stream = true;
    }
    // twiddles w[m] = exp(-2 pi i m / N), built in double
    std::vector<double> twd(2 * (size_t)N);
    for (int m = 0; m < N; ++m) {
        const double a = 2.0 * M_PI * (double)m / (double)N;
        twd[2 * m] = std::cos(a);
        twd[2 * m + 1] = -std::sin(a);
    }
    cudaError_t e = cudaSuccess;
    if (h->creal == 8) {
        std::vector<float> twf(2 * (size_t)N);
        for (size_t i = 0; i < twf.size(); ++i) twf[i] = (float)twd[i];
        e = cudaMemcpy(h->tw, twf.data(), twf.size() * sizeof(float), cudaMemcpyHostToDevice);
    } else {
        e = cudaMemcpy(h->tw, twd.data(), twd.size() * sizeof(double), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && nb > 1)
        e = cudaMemcpy(h->nu_box, nu_host, sizeof(double) * nb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->err, 0, 4 * sizeof(int), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->U, 0, nb * 3 * g.sS * h->creal, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->U0, 0, nb * 3 * g.sS * h->cacc, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->U1, 0, nb * 3 * g.sS * h->cacc, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->Om, 0, nb * 3 * g.sS * h->creal, h->stream);
    for (int v = 0; v < dns::PassSet::NCOLV && e == cudaSuccess; ++v)
        if (h->ps.prep_col[v]) e = h->ps.prep_col[v]();
    for (int v = 0; v < dns::PassSet::NP3V && e == cudaSuccess; ++v)
        if (h->ps.prep_p3[v]) e = h->ps.prep_p3[v]();
    for (int v = 0; v < dns::PassSet::NP5F && e == cudaSuccess; ++v)
        if (h->ps.prep_p5f[v]) e = h->ps.prep_p5f[v]();
    if (e == cudaSuccess) e = h->ps.prep_misc();
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        g_last_cuda = e;
        release(h);
        return DNS_ERR_CUDA;
    }
    *out = h;
    return DNS_OK;
}

// --------------------------------------------------------------- API
extern "C" {

const char *dns_strerror(int status) {
    switch (status) {
        case DNS_OK: return "ok";
        case DNS_ERR_ARG: return "invalid argument";
        case DNS_ERR_OOM: return "out of memory";
        case DNS_ERR_CUDA: return "CUDA error";
        case DNS_ERR_TIMEOUT: return "bounded device wait timed out";
        case DNS_ERR_NONFINITE: return "non-finite value in the state";
        case DNS_ERR_UNSUPPORTED: return "unsupported size, dtype or option";
        case DNS_ERR_GUARD: return "a guard region around a device buffer was overwritten";
        case DNS_ERR_INDEX: return "a kernel of the index-checked build met an address outside every buffer";
        default: return "unknown status";
    }
}

const char *dns_last_cuda_error(void) { return cudaGetErrorString(g_last_cuda); }

int dns_init(int N, double nu, double dt, int dtype, void *cuda_stream, dns_handle *out) {
    if (!out) return DNS_ERR_ARG;
    *out = nullptr;
    return ctx_create(N, 1, &nu, dt, dtype, (cudaStream_t)cuda_stream, out);
}

int dns_free(dns_handle h) {
    if (!h) return DNS_OK;
    cudaStreamSynchronize(h->stream);
    release(h);
    return DNS_OK;
}

int dns_check_guards(dns_handle h) {
    if (!h) return DNS_ERR_ARG;
    for (cudaStream_t st : {h->stream, h->s_in, h->s_out})
        if (st && cudaStreamSynchronize(st) != cudaSuccess) return DNS_ERR_CUDA;
    return check_guards(h);
}

// After the stream has drained: DNS_ERR_TIMEOUT if a kernel gave up a
// bounded wait (the word stays set; the state is then not trustworthy).
static int poll_device_status(dns_ctx *h) {
    int v = 0;
    CK(cudaMemcpy(&v, h->err, sizeof(int), cudaMemcpyDeviceToHost));
    return v == 0 ? DNS_OK : (v == dns::kErrIndex ? DNS_ERR_INDEX : DNS_ERR_TIMEOUT);
}

int dns_synchronize(dns_handle h) {
    TraceRange trace_("dns_synchronize");
    if (!h) return DNS_ERR_ARG;
    CK(cudaStreamSynchronize(h->stream));
    if (h->s_in) CK(cudaStreamSynchronize(h->s_in));
    if (h->s_out) CK(cudaStreamSynchronize(h->s_out));
    return poll_device_status(h);
}

}  // extern "C"

// The device side of the failure detection, exercised on purpose: one thread
// arms an mbarrier that nothing will ever complete and waits on it with the
// same bounded wait the bulk-copy consumers use, for limit_ns; the wait gives
// up, the code goes to the handle's status word and the kernel returns.  No
// copy is in flight, so nothing is left behind.
__global__ void k_wait_timeout_check(int *err, unsigned long long limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        dns::mbar_init(&bar, 1);
        if (!dns::mbar_wait_bounded(&bar, 0, limit_ns)) dns::record_error(err, dns::kErrWaitTimeout);
    }
}

extern "C" int dns_check_wait_timeout(dns_handle h, double seconds) {
    if (!h || !(seconds > 0.0) || !(seconds <= 2.0)) return DNS_ERR_ARG;
    k_wait_timeout_check<<<1, 32, 0, h->stream>>>(h->err, (unsigned long long)(seconds * 1e9));
    CK(cudaGetLastError());
    return DNS_OK;
}

// The index check exercised on purpose: one thread hands the check the
// address one byte past the end of buffer B.  The check compares addresses
// only; nothing is read or written there, and the check records the
// rejected address and this source line in the status word.
__global__ void k_index_check_selftest(dns::Chk ck, const unsigned char *probe) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const bool ok = DNS_RANGE_OK(ck, probe, 1);
        (void)ok;
    }
}

extern "C" int dns_checked_build(void) {
#ifdef DNS_CHECKED
    return 1;
#else
    return 0;
#endif
}

extern "C" int dns_check_index_selftest(dns_handle h) {
    if (!h) return DNS_ERR_ARG;
#ifdef DNS_CHECKED
    const unsigned char *end = static_cast<const unsigned char *>(h->B) + (size_t)h->g.nb * 6 * h->g.sB * h->creal;
    k_index_check_selftest<<<1, 32, 0, h->stream>>>(h->g.chk(), end);
    CK(cudaGetLastError());
    return DNS_OK;
#else
    return DNS_ERR_UNSUPPORTED;
#endif
}

extern "C" int dns_first_bad_access(dns_handle h, int *line, unsigned long long *address) {
    if (!h || !line || !address) return DNS_ERR_ARG;
    CK(cudaStreamSynchronize(h->stream));
    int w[4] = {0, 0, 0, 0};
    CK(cudaMemcpy(w, h->err, sizeof(w), cudaMemcpyDeviceToHost));
    unsigned long long a = 0;
    std::memcpy(&a, w + 2, sizeof(a));
    *line = w[0] == dns::kErrIndex ? w[1] : 0;
    *address = w[0] == dns::kErrIndex ? a : 0ull;
    return DNS_OK;
}

// Streams, events and staging buffers of the asynchronous host I/O, made on
// first use; a failure leaves none of them behind.
static void drop_async_io(dns_ctx *h) {
    for (cudaStream_t *st : {&h->s_in, &h->s_out})
        if (*st) {
            cudaStreamSynchronize(*st);
            cudaStreamDestroy(*st);
            *st = nullptr;
        }
    for (cudaEvent_t *ev : {&h->in_copied, &h->in_free, &h->out_ready[0], &h->out_ready[1], &h->out_copied[0],
                            &h->out_copied[1]})
        if (*ev) {
            cudaEventDestroy(*ev);
            *ev = nullptr;
        }
    for (void **p : {&h->io_in, &h->io_out[0], &h->io_out[1]})
        if (*p) {
            dev_free(h, *p);
            *p = nullptr;
        }
}

static int ensure_async_io(dns_ctx *h) {
    if (h->io_out[1]) return DNS_OK;  // the last thing made: all of it exists
    const size_t bytes = 3ull * h->N * h->N * (h->N / 2 + 1) * h->cio;
    cudaError_t e = cudaSuccess;
    for (cudaStream_t *st : {&h->s_in, &h->s_out})
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(st, cudaStreamNonBlocking);
    for (cudaEvent_t *ev : {&h->in_copied, &h->in_free, &h->out_ready[0], &h->out_ready[1], &h->out_copied[0],
                            &h->out_copied[1]})
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        g_last_cuda = e;
        drop_async_io(h);
        return DNS_ERR_CUDA;
    }
    for (void **p : {&h->io_in, &h->io_out[0], &h->io_out[1]}) {
        const int rc = dev_alloc(h, p, bytes);
        if (rc != DNS_OK) {
            drop_async_io(h);
            return rc;
        }
    }
    return DNS_OK;
}

extern "C" {

int dns_set_velocity_async(dns_handle h, const void *uhat) {
    TraceRange trace_("dns_set_velocity_async");
    if (!h || !uhat) return DNS_ERR_ARG;
    const int rc = ensure_async_io(h);
    if (rc != DNS_OK) return rc;
    const size_t bytes = 3ull * h->N * h->N * (h->N / 2 + 1) * h->cio;
    // the staging buffer is free once the previous conversion has read it
    CK(cudaStreamWaitEvent(h->s_in, h->in_free, 0));
    CK(cudaMemcpyAsync(h->io_in, uhat, bytes, cudaMemcpyHostToDevice, h->s_in));
    CK(cudaEventRecord(h->in_copied, h->s_in));
    CK(cudaStreamWaitEvent(h->stream, h->in_copied, 0));
    CK(full_to_state(h, h->io_in, h->U, h->U0));
    CK(cudaEventRecord(h->in_free, h->stream));
    CK(curl_box(h, 0));
    return DNS_OK;
}

int dns_get_velocity_async(dns_handle h, void *uhat) {
    TraceRange trace_("dns_get_velocity_async");
    if (!h || !uhat) return DNS_ERR_ARG;
    const int rc = ensure_async_io(h);
    if (rc != DNS_OK) return rc;
    const size_t bytes = 3ull * h->N * h->N * (h->N / 2 + 1) * h->cio;
    const int k = h->out_slot;
    h->out_slot ^= 1;
    // this slot's previous read-back (two calls ago) must have left it
    CK(cudaStreamWaitEvent(h->stream, h->out_copied[k], 0));
    CK(acc_to_full(h, h->U0, h->io_out[k]));
    CK(cudaEventRecord(h->out_ready[k], h->stream));
    CK(cudaStreamWaitEvent(h->s_out, h->out_ready[k], 0));
    CK(cudaMemcpyAsync(uhat, h->io_out[k], bytes, cudaMemcpyDeviceToHost, h->s_out));
    CK(cudaEventRecord(h->out_copied[k], h->s_out));
    return DNS_OK;
}

int dns_set_velocity(dns_handle h, const void *uhat, int on_device) {
    TraceRange trace_("dns_set_velocity");
    if (!h || !uhat) return DNS_ERR_ARG;
    return set_state(h, 0, uhat, on_device);
}

int dns_set_velocity_physical(dns_handle h, const void *u, int on_device) {
    TraceRange trace_("dns_set_velocity_physical");
    if (!h || !u) return DNS_ERR_ARG;
    const size_t nreal = 3ull * h->N * h->N * h->N;
    const size_t bytes = nreal * (h->cio / 2);
    const void *src = u;
    if (!on_device) {
        CK(cudaMemcpyAsync(h->io, u, bytes, cudaMemcpyHostToDevice, h->stream));
        src = h->io;
    } else {
        refresh_ranges(h, u, bytes);
    }
    CK(h->ps.zfwd(h->g, h->tw, src, h->B, h->stream));
    CK(h->ps.p4[h->plan[3]](h->g, h->tw, h->B, h->A, h->stream));
    dns::UpdateArgsErased a{};
    a.dU = h->rout;
    a.stage = -2;
    CK(launch_back(h, h->g, a, no_mark));
    const long long n = 3 * h->g.sS;
    CK(cudaMemcpyAsync(h->U0, h->rout, (size_t)n * h->cacc, cudaMemcpyDeviceToDevice, h->stream));
    if (h->same_type) {
        CK(cudaMemcpyAsync(h->U, h->rout, (size_t)n * h->cacc, cudaMemcpyDeviceToDevice, h->stream));
    } else {
        k_convert<double2, float2><<<grid_for(n), 256, 0, h->stream>>>((const double2 *)h->rout, (float2 *)h->U, n,
                                                                        h->g.chk());
        CK(cudaGetLastError());
    }
    CK(curl_box(h, 0));
    CK(cudaStreamSynchronize(h->stream));
    if (on_device) refresh_ranges(h);
    return DNS_OK;
}

int dns_get_velocity(dns_handle h, void *uhat, int on_device) {
    TraceRange trace_("dns_get_velocity");
    if (!h || !uhat) return DNS_ERR_ARG;
    return get_state(h, 0, uhat, on_device);
}

int dns_rhs(dns_handle h, const void *uhat_in, void *duhat_out, int on_device) {
    TraceRange trace_("dns_rhs");
    if (!h || !uhat_in || !duhat_out) return DNS_ERR_ARG;
    const size_t bytes = 3ull * h->N * h->N * (h->N / 2 + 1) * h->cio;
    const void *src = uhat_in;
    if (!on_device) {
        CK(cudaMemcpyAsync(h->io, uhat_in, bytes, cudaMemcpyHostToDevice, h->stream));
        src = h->io;
    } else {
        refresh_ranges(h, uhat_in, bytes, duhat_out, bytes);
    }
    CK(full_to_state(h, src, h->rin, nullptr));
    Geo g1 = h->g;
    g1.nb = 1;
    CK(h->ps.curl(g1, h->rin, h->rom, h->stream));
    CK(launch_front(h, h->rin, h->rom));
    dns::UpdateArgsErased a{};
    a.U = h->rin;
    a.dU = h->rout;
    a.nu = h->nu;
    a.stage = -1;
    if (h->closure) {
        CK(dns::les_closure_forcing(h->closure, h->g, h->rin, h->Fext, h->stream));
        a.Fext = h->Fext;
    }
    CK(launch_back(h, h->g, a, no_mark));
    if (on_device) {
        CK(acc_to_full(h, h->rout, duhat_out));
    } else {
        CK(acc_to_full(h, h->rout, h->io));
        CK(cudaMemcpyAsync(duhat_out, h->io, bytes, cudaMemcpyDeviceToHost, h->stream));
    }
    CK(cudaStreamSynchronize(h->stream));
    if (on_device) refresh_ranges(h);
    return DNS_OK;
}

int dns_step(dns_handle h, int n) {
    TraceRange trace_("dns_step");
    if (!h || n < 0) return DNS_ERR_ARG;
    if (n == 0) return DNS_OK;
    if (!h->exec) {
        CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = enqueue_step(h, nullptr);
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(h->stream, &graph);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            g_last_cuda = e != cudaSuccess ? e : e2;
            cudaGetLastError();
            return DNS_ERR_CUDA;
        }
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(graph);
            g_last_cuda = e;
            return DNS_ERR_CUDA;
        }
        h->graph = graph;
        h->exec = exec;
    }
    for (int i = 0; i < n; ++i) CK(cudaGraphLaunch(h->exec, h->stream));
    h->t += n * h->dt;
    h->step += n;
    return DNS_OK;
}

int dns_step_profiled(dns_handle h, int n, double *pass_ms, double *total_ms) {
    TraceRange trace_("dns_step_profiled");
    if (!h || n < 0 || !pass_ms) return DNS_ERR_ARG;
    for (int i = 0; i < DNS_NPASS; ++i) pass_ms[i] = 0.0;
    if (total_ms) *total_ms = 0.0;
    if (n == 0) return DNS_OK;
    const int per = 4 * DNS_NPASS;
    std::vector<cudaEvent_t> ev((size_t)per * n + 1, nullptr);
    int rc = DNS_OK;
    for (auto &x : ev)
        if (cudaEventCreate(&x) != cudaSuccess) {
            x = nullptr;
            rc = DNS_ERR_CUDA;
        }
    if (!rc && cudaEventRecord(ev[0], h->stream) != cudaSuccess) rc = DNS_ERR_CUDA;
    for (int i = 0; i < n && !rc; ++i) {
        cudaError_t e = enqueue_step(h, ev.data() + (size_t)per * i);
        if (e != cudaSuccess) {
            g_last_cuda = e;
            rc = DNS_ERR_CUDA;
        }
    }
    if (!rc && cudaStreamSynchronize(h->stream) != cudaSuccess) rc = DNS_ERR_CUDA;
    if (!rc) {
        for (size_t i = 0; i + 1 < ev.size(); ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
            pass_ms[i % DNS_NPASS] += ms;
        }
        float tot = 0.f;
        cudaEventElapsedTime(&tot, ev[0], ev.back());
        if (total_ms) *total_ms = tot;
        h->t += n * h->dt;
        h->step += n;
    }
    for (auto &x : ev)
        if (x) cudaEventDestroy(x);
    return rc;
}

static int stats_sums(dns_handle h, double *se, double *sd) { return stats_sums_box(h, 0, se, sd); }

int dns_energy(dns_handle h, double *E) {
    if (!h || !E) return DNS_ERR_ARG;
    double se, sd;
    int rc = stats_sums(h, &se, &sd);
    if (rc) return rc;
    const double N3 = (double)h->N * h->N * h->N;
    *E = se / (2.0 * N3 * N3);
    return std::isfinite(*E) ? DNS_OK : DNS_ERR_NONFINITE;
}

int dns_dissipation(dns_handle h, double *eps) {
    if (!h || !eps) return DNS_ERR_ARG;
    double se, sd;
    int rc = stats_sums(h, &se, &sd);
    if (rc) return rc;
    const double N3 = (double)h->N * h->N * h->N;
    *eps = h->nu * sd / (N3 * N3);
    return std::isfinite(*eps) ? DNS_OK : DNS_ERR_NONFINITE;
}

int dns_spectrum(dns_handle h, double *Ek, int nshells) {
    if (!h || !Ek || nshells < 1) return DNS_ERR_ARG;
    if (h->dtype == DNS_F32)
        dns::k_spectrum<float><<<h->smax, 256, 0, h->stream>>>(h->g, (const float2 *)h->U0, h->Ek);
    else
        dns::k_spectrum<double><<<h->smax, 256, 0, h->stream>>>(h->g, (const double2 *)h->U0, h->Ek);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(h->host, h->Ek, sizeof(double) * h->smax, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (int s = 0; s < nshells; ++s) Ek[s] = s < h->smax ? h->host[s] : 0.0;
    return DNS_OK;
}

int dns_time(dns_handle h, double *t, long *step) {
    if (!h) return DNS_ERR_ARG;
    if (t) *t = h->t;
    if (step) *step = h->step;
    return DNS_OK;
}

int dns_set_time(dns_handle h, double t, long step) {
    if (!h || !std::isfinite(t) || step < 0) return DNS_ERR_ARG;
    h->t = t;
    h->step = step;
    return DNS_OK;
}

int dns_query(dns_handle h, int *N, int *dtype, int *kmax, double *nu, double *dt) {
    if (!h) return DNS_ERR_ARG;
    if (N) *N = h->N;
    if (dtype) *dtype = h->dtype;
    if (kmax) *kmax = h->g.K;
    if (nu) *nu = h->nu;
    if (dt) *dt = h->dt;
    return DNS_OK;
}

int dns_device_bytes(dns_handle h, long long *bytes) {
    if (!h || !bytes) return DNS_ERR_ARG;
    *bytes = h->bytes;
    return DNS_OK;
}

// --------------------------------------------------------------- autotuner
}  // extern "C"

static void drop_graph(dns_ctx *h) {
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->exec = nullptr;
    h->graph = nullptr;
}

static bool variant_exists(const dns_ctx *h, int pass, int v) {
    if (pass == 2) return v >= 0 && v < dns::PassSet::NP3V && h->ps.p3[v];
    if (pass < 0 || pass > 4) return false;
    if (pass == 4 && v >= dns::PassSet::NCOLV)
        return v < dns::PassSet::NCOLV + dns::PassSet::NP5F && h->ps.p5f[v - dns::PassSet::NCOLV];
    return v >= 0 && v < dns::PassSet::NCOLV && h->ps.p1[v];
}

static int variant_count(int pass) {
    if (pass == 2) return dns::PassSet::NP3V;
    return pass == 4 ? dns::PassSet::NCOLV + dns::PassSet::NP5F : dns::PassSet::NCOLV;
}

// Mean device time of `reps` launches of one variant of one pass on the
// handle's scratch buffers; the state is only read.  Pass 4 is timed
// together with the update it feeds (P5a + P5b, or the fused form) as a
// middle RK4 stage of the first box (the heaviest stage: it reads u, u0, u1
// and writes u1, the next input and its curl), with those three outputs
// redirected to the right-hand-side scratch buffers, so both forms compare
// on the work a step does.
static cudaError_t time_variant(dns_ctx *h, int pass, int v, int reps, float *ms) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const double scale = 1.0 / ((double)h->N * h->N * h->N);
    Geo g1 = h->g;
    g1.nb = 1;
    dns::UpdateArgsErased ra = stage_args(h, 1);
    ra.U = h->U;
    ra.U1 = h->rout;   // accumulator type, 3 fields of one box
    ra.Uout = h->rin;  // field type
    ra.Om = h->rom;    // field type
    ra.Fext = nullptr;
    ra.nu_box = nullptr;
    auto launch = [&]() -> cudaError_t {
        switch (pass) {
            case 0: return h->ps.p1[v](h->g, h->tw, h->U, h->Om, h->A, scale, h->stream);
            case 1: return h->ps.p2[v](h->g, h->tw, h->A, h->B, h->stream);
            case 2: return h->ps.p3[v](h->g, h->tw, h->B, h->stream);
            case 3: return h->ps.p4[v](h->g, h->tw, h->B, h->A, h->stream);
            default: {
                if (v >= dns::PassSet::NCOLV)
                    return h->ps.p5f[v - dns::PassSet::NCOLV](g1, h->tw, h->A, ra, h->stream);
                cudaError_t e2 = h->ps.p5a[v](g1, h->tw, h->A, h->B, h->stream);
                return e2 != cudaSuccess ? e2 : h->ps.p5b(g1, h->B, ra, h->stream);
            }
        }
    };
    if (e == cudaSuccess) e = launch();  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
    for (int i = 0; i < reps && e == cudaSuccess; ++i) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    *ms = t / reps;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return e;
}

static void device_name(char *out, size_t n) {
    int dev = 0;
    cudaDeviceProp prop;
    out[0] = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess) {
        size_t i = 0;
        for (; i + 1 < n && prop.name[i]; ++i) out[i] = prop.name[i] == '"' ? '\'' : prop.name[i];
        out[i] = 0;
    }
}

// Cache lines: {"gpu": "<name>", "N": n, "dtype": d, "nb": b, "plan": [p1, p2, p3, p4, p5a]}
static bool cache_lookup(const char *path, const char *gpu, const dns_ctx *h, int *plan) {
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    char line[1024];
    bool found = false;
    while (!found && std::fgets(line, sizeof line, f)) {
        static const char kGpuKey[] = "\"gpu\": \"";
        const char *g = std::strstr(line, kGpuKey);
        const char *q = std::strstr(line, "\"N\":");
        if (!g || !q) continue;
        g += sizeof(kGpuKey) - 1;
        const char *ge = std::strchr(g, '"');
        if (!ge || (size_t)(ge - g) != std::strlen(gpu) || std::strncmp(g, gpu, ge - g) != 0) continue;
        int N = 0, dt = 0, nb = 0, p[5];
        if (std::sscanf(q, "\"N\": %d, \"dtype\": %d, \"nb\": %d, \"plan\": [%d, %d, %d, %d, %d]", &N, &dt, &nb, &p[0],
                        &p[1], &p[2], &p[3], &p[4]) != 8)
            continue;
        if (N != h->N || dt != h->dtype || nb != h->g.nb) continue;
        bool ok = true;
        for (int i = 0; i < 5; ++i) ok = ok && variant_exists(h, i, p[i]);
        if (ok) {
            for (int i = 0; i < 5; ++i) plan[i] = p[i];
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

static int autotune_ctx(dns_ctx *h, const char *cache_path, int reps) {
    char gpu[256];
    device_name(gpu, sizeof gpu);
    int plan[5];
    if (cache_path && cache_lookup(cache_path, gpu, h, plan)) {
        for (int i = 0; i < 5; ++i) h->plan[i] = plan[i];
        drop_graph(h);
        return DNS_OK;
    }
    CK(cudaStreamSynchronize(h->stream));
    float best_ms[5];
    for (int pass = 0; pass < 5; ++pass) {
        int best = 0;
        float bt = 1e30f;
        for (int v = 0; v < variant_count(pass); ++v) {
            if (!variant_exists(h, pass, v)) continue;
            float ms = 0.f;
            CK(time_variant(h, pass, v, reps, &ms));
            if (ms < bt) {
                bt = ms;
                best = v;
            }
        }
        plan[pass] = best;
        best_ms[pass] = bt;
    }
    for (int i = 0; i < 5; ++i) h->plan[i] = plan[i];
    drop_graph(h);
    if (cache_path) {
        FILE *f = std::fopen(cache_path, "a");
        if (f) {
            std::fprintf(f,
                         "{\"gpu\": \"%s\", \"N\": %d, \"dtype\": %d, \"nb\": %d, \"plan\": [%d, %d, %d, %d, %d], "
                         "\"ms\": [%.4f, %.4f, %.4f, %.4f, %.4f]}\n",
                         gpu, h->N, h->dtype, h->g.nb, plan[0], plan[1], plan[2], plan[3], plan[4], best_ms[0],
                         best_ms[1], best_ms[2], best_ms[3], best_ms[4]);
            std::fclose(f);
        }
    }
    return DNS_OK;
}

extern "C" {

int dns_autotune(dns_handle h, const char *cache_path, int *plan_out) {
    TraceRange trace_("dns_autotune");
    if (!h) return DNS_ERR_ARG;
    int rc = autotune_ctx(h, cache_path, 3);
    if (!rc && plan_out)
        for (int i = 0; i < 5; ++i) plan_out[i] = h->plan[i];
    return rc;
}

int dns_set_integrator(dns_handle h, int kind) {
    if (!h || (kind != DNS_RK4 && kind != DNS_IFRK4)) return DNS_ERR_ARG;
    if (kind != h->integrator) {
        h->integrator = kind;
        drop_graph(h);
    }
    return DNS_OK;
}

int dns_les_set_closure_stages(dns_handle h, int every_stage) {
    if (!h || (every_stage != 0 && every_stage != 1)) return DNS_ERR_ARG;
    if (h->closure_every_stage != every_stage) {
        h->closure_every_stage = every_stage;
        drop_graph(h);  // the captured step holds the old choice
    }
    return DNS_OK;
}

int dns_get_plan(dns_handle h, int *plan) {
    if (!h || !plan) return DNS_ERR_ARG;
    for (int i = 0; i < 5; ++i) plan[i] = h->plan[i];
    return DNS_OK;
}

int dns_set_plan(dns_handle h, const int *plan) {
    if (!h || !plan) return DNS_ERR_ARG;
    for (int i = 0; i < 5; ++i)
        if (!variant_exists(h, i, plan[i])) return DNS_ERR_UNSUPPORTED;
    for (int i = 0; i < 5; ++i) h->plan[i] = plan[i];
    drop_graph(h);
    return DNS_OK;
}

int dns_variant_info(dns_handle h, int pass, int variant, int *lines, int *max_radix, int *threads) {
    if (!h || pass < 0 || pass > 4) return DNS_ERR_ARG;
    if (!variant_exists(h, pass, variant)) return DNS_ERR_UNSUPPORTED;
    if (pass == 2) {
        if (lines) *lines = h->ps.p3_l[variant];
        if (max_radix) *max_radix = h->ps.p3_r[variant];
        if (threads) *threads = h->ps.p3_t[variant];
    } else if (pass == 4 && variant >= dns::PassSet::NCOLV) {
        const int f = variant - dns::PassSet::NCOLV;
        if (lines) *lines = h->ps.p5f_w[f];
        if (max_radix) *max_radix = h->ps.p5f_r[f];
        if (threads) *threads = h->ps.p5f_t[f];
    } else {
        if (lines) *lines = h->ps.col_w[variant];
        if (max_radix) *max_radix = h->ps.col_r[variant];
        if (threads) *threads = h->ps.col_t[variant];
    }
    return DNS_OK;
}

// --------------------------------------------------------------- ensemble
}  // extern "C"

struct dns_ens_ctx {
    int nbox = 0, dtype = 0;
    double dt = 0, t = 0;
    long step = 0;
    std::vector<dns_ctx *> cls;    // one context per distinct N
    std::vector<int> box_cls, box_idx;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

static void ens_release(dns_ens_ctx *e) {
    if (!e) return;
    if (e->exec) cudaGraphExecDestroy(e->exec);
    if (e->graph) cudaGraphDestroy(e->graph);
    for (dns_ctx *c : e->cls) release(c);
    if (e->own_stream && e->stream) cudaStreamDestroy(e->stream);
    delete e;
}

extern "C" {

int dns_ensemble_init(int nbox, const int *N, const double *nu, double dt, int dtype, void *cuda_stream,
                      dns_ensemble *out) {
    if (!out) return DNS_ERR_ARG;
    *out = nullptr;
    if (nbox < 1 || !N || !nu) return DNS_ERR_ARG;
    if (dtype < DNS_F32 || dtype > DNS_F32_ACC64 || !(dt > 0.0) || !std::isfinite(dt)) return DNS_ERR_ARG;
    for (int b = 0; b < nbox; ++b) {
        if (!dns::getter_for(N[b])) return DNS_ERR_UNSUPPORTED;
        if (!(nu[b] > 0.0) || !std::isfinite(nu[b])) return DNS_ERR_ARG;
    }
    dns_ens_ctx *e = new (std::nothrow) dns_ens_ctx();
    if (!e) return DNS_ERR_OOM;
    e->nbox = nbox;
    e->dtype = dtype;
    e->dt = dt;
    if (cuda_stream) {
        e->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreate(&e->stream) != cudaSuccess) {
            delete e;
            return DNS_ERR_CUDA;
        }
        e->own_stream = true;
    }
    // group boxes by mesh size, in order of first appearance
    std::vector<int> sizes;
    e->box_cls.resize(nbox);
    e->box_idx.resize(nbox);
    std::vector<std::vector<double>> nus;
    for (int b = 0; b < nbox; ++b) {
        int c = -1;
        for (size_t i = 0; i < sizes.size(); ++i)
            if (sizes[i] == N[b]) c = (int)i;
        if (c < 0) {
            c = (int)sizes.size();
            sizes.push_back(N[b]);
            nus.emplace_back();
        }
        e->box_cls[b] = c;
        e->box_idx[b] = (int)nus[c].size();
        nus[c].push_back(nu[b]);
    }
    for (size_t c = 0; c < sizes.size(); ++c) {
        dns_ctx *h = nullptr;
        int rc = ctx_create(sizes[c], (int)nus[c].size(), nus[c].data(), dt, dtype, e->stream, &h);
        if (rc) {
            ens_release(e);
            return rc;
        }
        e->cls.push_back(h);
    }
    *out = e;
    return DNS_OK;
}

int dns_ensemble_free(dns_ensemble e) {
    if (!e) return DNS_OK;
    cudaStreamSynchronize(e->stream);
    ens_release(e);
    return DNS_OK;
}

int dns_ensemble_check_guards(dns_ensemble e) {
    if (!e) return DNS_ERR_ARG;
    if (cudaStreamSynchronize(e->stream) != cudaSuccess) return DNS_ERR_CUDA;
    for (dns_ctx *c : e->cls) {
        const int rc = dns_check_guards(c);
        if (rc != DNS_OK) return rc;
    }
    return DNS_OK;
}

int dns_ensemble_set_velocity(dns_ensemble e, int box, const void *uhat, int on_device) {
    if (!e || !uhat || box < 0 || box >= e->nbox) return DNS_ERR_ARG;
    return set_state(e->cls[e->box_cls[box]], e->box_idx[box], uhat, on_device);
}

int dns_ensemble_get_velocity(dns_ensemble e, int box, void *uhat, int on_device) {
    if (!e || !uhat || box < 0 || box >= e->nbox) return DNS_ERR_ARG;
    return get_state(e->cls[e->box_cls[box]], e->box_idx[box], uhat, on_device);
}

int dns_ensemble_step(dns_ensemble e, int n) {
    TraceRange trace_("dns_ensemble_step");
    if (!e || n < 0) return DNS_ERR_ARG;
    if (n == 0) return DNS_OK;
    if (!e->exec) {
        CK(cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t err = cudaSuccess;
        for (dns_ctx *h : e->cls)
            if (err == cudaSuccess) err = enqueue_step(h, nullptr);
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(e->stream, &graph);
        if (err != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            g_last_cuda = err != cudaSuccess ? err : e2;
            cudaGetLastError();
            return DNS_ERR_CUDA;
        }
        cudaGraphExec_t exec = nullptr;
        err = cudaGraphInstantiate(&exec, graph, 0);
        if (err != cudaSuccess) {
            cudaGraphDestroy(graph);
            g_last_cuda = err;
            return DNS_ERR_CUDA;
        }
        e->graph = graph;
        e->exec = exec;
    }
    for (int i = 0; i < n; ++i) CK(cudaGraphLaunch(e->exec, e->stream));
    e->t += n * e->dt;
    e->step += n;
    return DNS_OK;
}

int dns_ensemble_synchronize(dns_ensemble e) {
    if (!e) return DNS_ERR_ARG;
    CK(cudaStreamSynchronize(e->stream));
    for (dns_ctx *c : e->cls) {
        const int rc = poll_device_status(c);
        if (rc) return rc;
    }
    return DNS_OK;
}

int dns_ensemble_energy(dns_ensemble e, double *E) {
    if (!e || !E) return DNS_ERR_ARG;
    int status = DNS_OK;
    for (int b = 0; b < e->nbox; ++b) {
        dns_ctx *h = e->cls[e->box_cls[b]];
        double se, sd;
        int rc = stats_sums_box(h, e->box_idx[b], &se, &sd);
        if (rc) return rc;
        const double N3 = (double)h->N * h->N * h->N;
        E[b] = se / (2.0 * N3 * N3);
        if (!std::isfinite(E[b])) status = DNS_ERR_NONFINITE;
    }
    return status;
}

int dns_ensemble_time(dns_ensemble e, double *t, long *step) {
    if (!e) return DNS_ERR_ARG;
    if (t) *t = e->t;
    if (step) *step = e->step;
    return DNS_OK;
}

int dns_ensemble_autotune(dns_ensemble e, const char *cache_path) {
    if (!e) return DNS_ERR_ARG;
    for (dns_ctx *h : e->cls) {
        int rc = autotune_ctx(h, cache_path, 3);
        if (rc) return rc;
    }
    if (e->exec) cudaGraphExecDestroy(e->exec);
    if (e->graph) cudaGraphDestroy(e->graph);
    e->exec = nullptr;
    e->graph = nullptr;
    return DNS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- internal accessors (LES unit)
namespace dns {
int internal_view(dns_handle h, InternalView *v) {
    if (!h || !v) return DNS_ERR_ARG;
    v->N = h->N;
    v->dtype = h->dtype;
    v->g = h->g;
    v->U0 = h->U0;
    v->stream = h->stream;
    return DNS_OK;
}

int internal_set_closure(dns_handle h, LesClosure *c) {
    if (!h) return DNS_ERR_ARG;
    if (h->closure) les_closure_release(h->closure);
    h->closure = c;
    if (c && !h->Fext) {
        const int rc = dev_alloc(h, &h->Fext, 3 * h->g.sS * h->creal);
        if (rc != DNS_OK) {
            h->Fext = nullptr;
            h->closure = nullptr;
            les_closure_release(c);
            return rc;
        }
    }
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    h->exec = nullptr;
    h->graph = nullptr;
    return DNS_OK;
}
}  // namespace dns
