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
    double nu, adt, bdt;
    const double *nu_box;  // per-box viscosity for batched boxes, or nullptr
    int stage;  // 0..3 RK4 stage, -1 right-hand side only, -2 raw forward transform
};

// Launch shapes and entry points for one (N, dtype).  `real` is the field
// type (float or double); `acc` the RK4 state type.
struct PassSet {
    int W, T;    // P1, P2, P4, P5a: columns per tile, threads
    int L3, T3;  // P3: lines per block, threads
    size_t smem_col, smem_p3;
    cudaError_t (*p1)(const Geo &, const void *tw, const void *U, const void *Om, void *A, double scale,
                      cudaStream_t);
    // Om = i k x U on the stored modes (all boxes of the context)
    cudaError_t (*curl)(const Geo &, const void *U, void *Om, cudaStream_t);
    cudaError_t (*p2)(const Geo &, const void *tw, const void *A, void *B, cudaStream_t);
    cudaError_t (*p3)(const Geo &, const void *tw, void *B, cudaStream_t);
    cudaError_t (*p4)(const Geo &, const void *tw, const void *B, void *A, cudaStream_t);
    cudaError_t (*p5a)(const Geo &, const void *tw, const void *A, void *Nh, cudaStream_t);
    cudaError_t (*p5b)(const Geo &, const void *Nh, const UpdateArgsErased &, cudaStream_t);
    // physical real lines [3][N][N][N] (io real type) -> B fields 0..2, kz <= K
    cudaError_t (*zfwd)(const Geo &, const void *tw, const void *u, void *B, cudaStream_t);
    // raise shared-memory limits of all kernels above; call before any launch
    cudaError_t (*prepare)();
};

// dtype: 0 = F32, 1 = F64, 2 = F32_ACC64.  io_double: physical input type.
typedef bool (*PassGetter)(int dtype, PassSet *out);

}  // namespace dns
