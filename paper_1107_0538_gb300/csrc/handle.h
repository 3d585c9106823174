// The solver handle behind the opaque cg_handle of gbcg.h, shared by the
// translation units of the library (host code only; device code is in the
// .cu files).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <vector>

#include "cg_device.cuh"
#include "gbcg.h"
#include "sell.cuh"

namespace gbcg {
using SolveKernel = void (*)(Params);
struct LearnCtx;  // learned-preconditioner workspace (learn.cu)
}  // namespace gbcg

struct cg_handle {
    int device = 0;
    cudaStream_t stream = nullptr;
    cg_opts opts{};
    int32_t n = 0;
    int64_t nnz = 0;
    int ctas = 0;
    int ntiles = 0;
    int rpt = 0;                      // rows per thread kept in registers (0: none)
    gbcg::SolveKernel kernel = nullptr;
    int max_tile_nnz = 0;
    int evict_first = 0;
    int64_t device_bytes = 0;
    // device arrays
    int32_t *rowptr = nullptr, *colidx = nullptr, *cta_tile = nullptr, *cta_row = nullptr;
    int4 *tiles = nullptr, *segs = nullptr;
    uint16_t *lcol = nullptr;
    int window_tiles = 0;
    // mixed precision
    float *vals32 = nullptr, *diag_lo = nullptr, *dinv32 = nullptr;
    uint16_t *vals16 = nullptr;
    float *r32 = nullptr, *z32 = nullptr, *p32 = nullptr, *q32 = nullptr, *d32 = nullptr;
    float *pd32 = nullptr;            // inner direction of the mixed-precision solve
    double *vals = nullptr, *dinv = nullptr;
    double *r = nullptr, *z = nullptr, *p0 = nullptr, *q = nullptr;
    double *pd = nullptr;             // direction of the FP64 CG in memory mode
    double *partials = nullptr, *b_dev = nullptr, *x_dev = nullptr;
    unsigned int *bar = nullptr;
    gbcg::DevStatus *st = nullptr;
    gbcg::DevStatus *st_host = nullptr;  // pinned
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<void *> allocs;
    gbcg::LearnCtx *learn = nullptr;  // set by cg_set_learned
    // SELL-32 copy of the matrix (stand-alone and flexible-CG SpMV)
    long long *sell_ptr = nullptr;
    double *sell_vals = nullptr;
    int16_t *sell_c16 = nullptr;
    int32_t *sell_c32 = nullptr;
    int32_t sell_slices = 0;
    int sell_grid = 0;                // CTAs of a SELL SpMV launch
    int sell_solve = 0;               // 1: FP64 solves run cg_sell_kernel
    int sell_mem = 0;                 // 1: FP64 solves run cg_sellmem_kernel (vectors in memory)
    int32_t *sell_cut = nullptr;      // ctas + 1 slice boundaries of the slice kernel's CTAs
    int32_t *sell_split = nullptr;    // per slice: local block width (split layout), or nullptr
    void *sell_lo = nullptr;          // low-precision off-diagonals in the SELL layout (float or
                                      // BF16 bits, per opts.inner_values), or nullptr
};

namespace gbcg {

inline int cuda_fail(cudaError_t e) { return e == cudaErrorMemoryAllocation ? CG_ENOMEM : CG_ECUDA; }

// cudaMalloc recorded in the handle (freed with it).
template <class T>
int dev_alloc(cg_handle *h, T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    void *v = nullptr;
    cudaError_t e = cudaMalloc(&v, count * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(e);
    h->allocs.push_back(v);
    h->device_bytes += (int64_t)(count * sizeof(T));
    *p = static_cast<T *>(v);
    return CG_OK;
}

// An NVTX range over one library call (named "gbcg.<call>"), visible to
// Nsight tools; without a tool attached it costs a branch.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Kernel parameters of the handle's matrix, tiles and workspace (gbcg.cu).
Params base_params(const cg_handle *h);
// The handle's SELL-32 matrix.
inline SellMatrix sell_of(const cg_handle *h) {
    return SellMatrix{h->n,        h->sell_slices, h->evict_first, h->sell_ptr,
                      h->sell_vals, h->sell_c16,    h->sell_c32,     h->sell_split};
}
// Enqueues one persistent FP64 CG solve with the given preconditioner flag
// (0 plain, 1 Jacobi) on the handle's stream, without synchronizing (gbcg.cu).
int enqueue_fp64_solve(cg_handle *h, const double *b, double *x, double tol, int32_t maxit, int precond);
// Enqueues y = A x (SELL-32 SpMV) on the handle's stream (gbcg.cu).
int enqueue_spmv(cg_handle *h, const double *x, double *y);
// Flexible CG with the learned preconditioner (learn.cu).
int learn_solve(cg_handle *h, const double *b, double *x, double tol, int32_t maxit, cg_info *info);
// Frees the learned-preconditioner workspace of a handle (learn.cu).
void learn_free(cg_handle *h);
// Index faults counted by the bounds-check build in batch.cu and learn.cu
// (-1 in a normal build).
long long bounds_faults_batch();
long long bounds_faults_learn();

}  // namespace gbcg
