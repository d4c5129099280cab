// Internal interface between the C-ABI layer and the per-N kernel units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace dns {

struct Geo;

// Type-erased arguments of the update pass (see UpdateArgs in dns_passes.cuh).
struct UpdateArgsErased {
    const void *U, *U0;
    void *U1, *Uout, *U0out, *dU;
    void *Om;  // curl of the next stage input out, or nullptr
    const void *Fext;  // forcing added to the nonlinear term before the projection, or nullptr
    double nu, adt, bdt, dt;
    const double *nu_box;  // per-box viscosity for batched boxes, or nullptr
    int stage;  // 0..3 RK4 stage, -1 right-hand side only, -2 raw forward transform
    int ifrk;   // 1: integrating-factor RK4
};

typedef cudaError_t (*ColP1)(const Geo &, const void *tw, const void *U, const void *Om, void *A, double scale,
                             cudaStream_t);
typedef cudaError_t (*ColPass)(const Geo &, const void *tw, const void *src, void *dst, cudaStream_t);
typedef cudaError_t (*ZPass)(const Geo &, const void *tw, void *B, cudaStream_t);
typedef cudaError_t (*Prep)();
typedef cudaError_t (*P5Fused)(const Geo &, const void *tw, const void *A, const UpdateArgsErased &, cudaStream_t);

// Entry points for one (N, dtype): every compiled variant of each tuned pass
// (nullptr where a shape is not compiled) and the untuned kernels.
struct PassSet {
    static constexpr int NCOLV = 10;  // column-pass variants (W, RC, input by threads or bulk copy)
    static constexpr int NP3V = 16;   // z-pass variants (L, R3, resident blocks, input feed; the last two: one warp per line)
    ColP1 p1[NCOLV] = {};
    ColPass p2[NCOLV] = {}, p4[NCOLV] = {}, p5a[NCOLV] = {};
    Prep prep_col[NCOLV] = {};
    int col_w[NCOLV] = {}, col_r[NCOLV] = {}, col_t[NCOLV] = {};
    ZPass p3[NP3V] = {};
    Prep prep_p3[NP3V] = {};
    int p3_l[NP3V] = {}, p3_r[NP3V] = {}, p3_t[NP3V] = {};
    cudaError_t (*p5b)(const Geo &, const void *Nh, const UpdateArgsErased &, cudaStream_t) = nullptr;
    // fused P5a + P5b variants; plan[4] = NCOLV + v selects p5f[v]
    static constexpr int NP5F = 2;
    P5Fused p5f[NP5F] = {};
    Prep prep_p5f[NP5F] = {};
    int p5f_w[NP5F] = {}, p5f_r[NP5F] = {}, p5f_t[NP5F] = {};
    // physical real lines [3][N][N][N] (io real type) -> B fields 0..2, kz <= K
    cudaError_t (*zfwd)(const Geo &, const void *tw, const void *u, void *B, cudaStream_t) = nullptr;
    // Om = i k x U on the stored modes (all boxes of the context)
    cudaError_t (*curl)(const Geo &, const void *U, void *Om, cudaStream_t) = nullptr;
    Prep prep_misc = nullptr;
};

// dtype: 0 = F32, 1 = F64, 2 = F32_ACC64.
typedef bool (*PassGetter)(int dtype, PassSet *out);

// Learned-closure hook of an LES handle (implemented in dns_les.cu): from the
// stage input U (compact, FP32, one box) compute the forcing -i k_j tau_ij^
// on the stored modes into Fext (compact, 3 fields), on `stream`.
struct LesClosure;
cudaError_t les_closure_forcing(LesClosure *c, const Geo &g, const void *U, void *Fext, cudaStream_t stream);
void les_closure_release(LesClosure *c);
}  // namespace dns

#include "dns.h"
#include "dns_passes.cuh"

namespace dns {
// What the LES unit needs to see of a handle (defined in dns_api.cu).
struct InternalView {
    int N, dtype;
    Geo g;
    const void *U0;
    cudaStream_t stream;
};
int internal_view(dns_handle h, InternalView *v);
// Attach (or, with nullptr, detach) a closure; the handle takes ownership.
int internal_set_closure(dns_handle h, LesClosure *c);

}  // namespace dns
