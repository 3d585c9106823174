// cg_solve_noalloc: the FP64 CG solve for callers that cannot allocate
// device memory.
//
// Some callers of this library may not call cudaMalloc: code embedded in a
// framework whose caching allocator owns the device memory (a cudaMalloc
// beside it can fail once the framework holds the memory, and it
// synchronizes the whole device), real-time loops whose latency budget has no
// room for the device-wide synchronization an allocation implies, and
// plug-ins that run inside a host application with a fixed device-memory
// budget.  cg_create allocates the matrix copy and the solver workspace, so
// those callers cannot use it.  This entry point takes the matrix and the
// vectors from the caller and keeps its workspace (three vectors, the
// per-CTA partial sums, the grid-barrier counter and the status block) in one
// file-scope __device__ array of fixed size, so it allocates nothing, on the
// device or on the host.  It is synchronous: it returns once the result and
// the status are back.
//
// The workspace array is shared by every call in the process and keeps the
// contents of the last call: each call clears what must start at zero (the
// barrier counter and the status block) and writes every vector entry before
// reading it.  Two calls whose work overlaps on the GPU (on different streams,
// or from different host threads) race on that array.
//
// In host code the array's name only stands for it: its device address is
// looked up with cudaGetSymbolAddress, once per device, with that device
// current, on the device's first call.  With lazy module loading (the CUDA
// default) that first call is also what loads this module on the device and
// so creates the array; make it before any stream capture.  cudaDeviceReset
// destroys the array with the context, so the cached address is stale after
// it: a process that resets a device must not call this entry point on it
// again.
//
// It is a variant of cg_solve_kernel: the same recurrence, fixed-order
// reductions, thread-0 scalars and bounded grid barriers, with a plain
// row-per-thread SpMV straight from the caller's CSR arrays instead of the
// TMA-staged tiles (whose plan cg_create builds on the host).
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "cg_device.cuh"
#include "gbcg.h"

using namespace gbcg;

namespace {

constexpr int kNoallocMaxCtas = 256;
constexpr size_t kVecBytes = sizeof(double) * (size_t)CG_NOALLOC_MAX_N;
constexpr size_t kPartialBytes = sizeof(double) * 2 * kNoallocMaxCtas * kRedSlots;
constexpr size_t kOffR = 0;
constexpr size_t kOffP = kOffR + kVecBytes;
constexpr size_t kOffQ = kOffP + kVecBytes;
constexpr size_t kOffPartials = kOffQ + kVecBytes;
constexpr size_t kOffBar = kOffPartials + kPartialBytes;
constexpr size_t kOffStatus = kOffBar + 256;
constexpr size_t kScratchBytes = kOffStatus + 256;
constexpr int kNoallocSmem = kThreads * 8 + 64 + 64;

}  // namespace

// The workspace (about 6 MiB); every GPU that loads the library holds it
// until the process exits.
static __device__ __align__(256) unsigned char g_cg_noalloc_scratch[kScratchBytes];

namespace {

struct NoallocArgs {
    int32_t n;
    const int32_t *rowptr;
    const int32_t *colidx;
    const double *vals;
    const double *b;
    double *x;
    double tol;
    int32_t maxit;
};

// y_i = sum_k vals[k] * v[colidx[k]] for one row; false if the row's range or
// a column is out of bounds (the entry is then skipped).
__device__ __forceinline__ double noalloc_row(const NoallocArgs &A, int i, const double *v, int64_t nnz,
                                              bool &bad) {
    const int k0 = A.rowptr[i], k1 = A.rowptr[i + 1];
    if (k0 < 0 || k1 < k0 || (int64_t)k1 > nnz) {
        bad = true;
        return 0.0;
    }
    double s0 = 0.0, s1 = 0.0;
    int k = k0;
    for (; k + 1 < k1; k += 2) {
        const int c0 = A.colidx[k], c1 = A.colidx[k + 1];
        const bool ok0 = (unsigned)c0 < (unsigned)A.n, ok1 = (unsigned)c1 < (unsigned)A.n;
        bad |= !ok0 || !ok1;
        const double x0 = ok0 ? v[c0] : 0.0, x1 = ok1 ? v[c1] : 0.0;
        s0 = fma(A.vals[k], x0, s0);
        s1 = fma(A.vals[k + 1], x1, s1);
    }
    if (k < k1) {
        const int c0 = A.colidx[k];
        const bool ok0 = (unsigned)c0 < (unsigned)A.n;
        bad |= !ok0;
        s0 = fma(A.vals[k], ok0 ? v[c0] : 0.0, s0);
    }
    return s0 + s1;
}

__global__ void __launch_bounds__(kThreads, 1) cg_noalloc_kernel(NoallocArgs A, Params P, int64_t nnz) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem S;
    S.stage = nullptr;
    S.mbar = nullptr;
    S.red = reinterpret_cast<double *>(smem_raw);
    S.bcast = S.red + kThreads;
    S.ctl = reinterpret_cast<int *>(S.bcast + 8);
    const int tid = threadIdx.x;
    const int G = (int)gridDim.x;
    const int row_lo = (int)((int64_t)A.n * blockIdx.x / G);
    const int row_hi = (int)((int64_t)A.n * (blockIdx.x + 1) / G);
    unsigned int epoch = 0;
    int set = 0;
    bool bad = false;
    int status = CG_OK, iters = 0;
    double rr = 0.0, bb = 0.0, rho = 0.0, bnorm = 0.0;

    // setup: r = b - A x, p = r; r.r, b.b (and any malformed row)
    double v[3] = {0.0, 0.0, 0.0};
    for (int i = row_lo + tid; i < row_hi; i += kThreads) {
        const double bi = A.b[i];
        const double ri = bi - noalloc_row(A, i, A.x, nnz, bad);
        P.r[i] = ri;
        P.p0[i] = ri;
        v[0] = fma(ri, ri, v[0]);
        v[1] = fma(bi, bi, v[1]);
    }
    v[2] = __syncthreads_or(bad) ? 1.0 : 0.0;
    block_sum<3>(v, S);
    publish_partials<3>(P, set, v);
    if (!grid_barrier(P, epoch, S)) return;
    {
        double t[3];
        grid_totals<3>(P, set, t);
        set ^= 1;
        if (tid == 0) {
            rr = t[0];
            bb = t[1];
            rho = t[0];
            bnorm = sqrt(bb);
            int go = 0, zero_b = 0;
            if (t[2] != 0.0) status = CG_EINVAL;
            else if (!finite_bits(bb) || !finite_bits(rr)) status = CG_ENAN;
            else if (bnorm == 0.0) { zero_b = 1; rr = 0.0; }
            else if (sqrt(rr) <= P.tol * bnorm) status = CG_OK;
            else go = 1;
            S.ctl[0] = go;
            S.ctl[2] = zero_b;
        }
        __syncthreads();
        if (S.ctl[2])
            for (int i = row_lo + tid; i < row_hi; i += kThreads) A.x[i] = 0.0;
    }
    if (S.ctl[0]) {
        if (tid == 0) status = CG_ENOCONV;
        for (int k = 1; k <= P.maxit; ++k) {
            // q = A p, p . q
            double pq = 0.0;
            for (int i = row_lo + tid; i < row_hi; i += kThreads) {
                const double qi = noalloc_row(A, i, P.p0, nnz, bad);
                P.q[i] = qi;
                pq = fma(P.p0[i], qi, pq);
            }
            double v1[1] = {pq};
            block_sum<1>(v1, S);
            publish_partials<1>(P, set, v1);
            if (!grid_barrier(P, epoch, S)) return;
            double sg[1];
            grid_totals<1>(P, set, sg);
            set ^= 1;
            if (tid == 0) {
                int go = 0;
                if (!finite_bits(sg[0])) status = CG_ENAN;
                else if (!(sg[0] > 0.0)) status = CG_EBREAKDOWN;
                else go = 1;
                S.bcast[0] = go ? rho / sg[0] : 0.0;
                S.ctl[0] = go;
            }
            __syncthreads();
            if (!S.ctl[0]) break;
            const double alpha = S.bcast[0];
            // x += alpha p, r -= alpha q; r.r
            double prr = 0.0;
            for (int i = row_lo + tid; i < row_hi; i += kThreads) {
                A.x[i] = fma(alpha, P.p0[i], A.x[i]);
                const double ri = fma(-alpha, P.q[i], P.r[i]);
                P.r[i] = ri;
                prr = fma(ri, ri, prr);
            }
            double v2[1] = {prr};
            block_sum<1>(v2, S);
            publish_partials<1>(P, set, v2);
            if (!grid_barrier(P, epoch, S)) return;
            double t2[1];
            grid_totals<1>(P, set, t2);
            set ^= 1;
            if (tid == 0) {
                iters = k;
                rr = t2[0];
                int go = 0;
                if (!finite_bits(rr)) status = CG_ENAN;
                else if (sqrt(rr) <= P.tol * bnorm) status = CG_OK;
                else if (!(rr > 0.0)) status = CG_EBREAKDOWN;
                else if (k < P.maxit) go = 1;
                if (go) {
                    S.bcast[1] = rr / rho;
                    rho = rr;
                }
                S.ctl[0] = go;
            }
            __syncthreads();
            if (!S.ctl[0]) break;
            const double beta = S.bcast[1];
            // p = r + beta p
            for (int i = row_lo + tid; i < row_hi; i += kThreads) P.p0[i] = fma(beta, P.p0[i], P.r[i]);
            if (!grid_barrier(P, epoch, S)) return;
        }
    }
    if (blockIdx.x == 0 && tid == 0) {
        P.st->iters = iters;
        P.st->rr = rr;
        P.st->bb = bb;
        P.st->true_rr = -1.0;
        atomicCAS(&P.st->status, 0, status);
    }
}

// Device address of the workspace, looked up once per device (with that
// device current) and cached; no allocation.
std::mutex g_setup_mutex;
unsigned char *g_scratch_ptr[128] = {};
int g_grid[128] = {};

int noalloc_setup(int dev, unsigned char **scratch, int *grid) {
    if (dev < 0 || dev >= 128) return CG_EINVAL;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_cg_noalloc_scratch) != cudaSuccess || !ptr) return CG_ECUDA;
        if (cudaFuncSetAttribute((const void *)cg_noalloc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kNoallocSmem) != cudaSuccess)
            return CG_ECUDA;
        int sms = 0, per_sm = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cg_noalloc_kernel, kThreads,
                                                          kNoallocSmem) != cudaSuccess ||
            per_sm < 1)
            return CG_ECUDA;
        int g = sms < kNoallocMaxCtas ? sms : kNoallocMaxCtas;
        g_grid[dev] = g;
        g_scratch_ptr[dev] = static_cast<unsigned char *>(ptr);
    }
    *scratch = g_scratch_ptr[dev];
    *grid = g_grid[dev];
    return CG_OK;
}

// True when p points into memory the current device can read in a kernel:
// a device allocation of that device, or managed memory.  Host memory
// (pageable or pinned) and other devices' allocations are refused before any
// launch.  cudaPointerGetAttributes allocates nothing.
bool on_device(const void *p, int dev) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();   // clear the (non-sticky) error recorded for an unknown pointer
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

int solve_noalloc(const cg_csr *A, const double *b, double *x, double tol, int32_t maxit, void *stream,
                  cg_info *info);

}  // namespace

// info->status is the return code whether or not the solve ran: a call
// rejected before the solve leaves a result with that status and nothing
// else (relres_true and reverted_at -1).
extern "C" int cg_solve_noalloc(const cg_csr *A, const double *b, double *x, double tol, int32_t maxit,
                                void *stream, cg_info *info) {
    constexpr int32_t kUnset = INT32_MIN;
    if (info) info->status = kUnset;
    const int rc = solve_noalloc(A, b, x, tol, maxit, stream, info);
    if (info) {
        if (info->status == kUnset) {
            *info = cg_info{};
            info->relres_true = -1.0;
            info->reverted_at = -1;
        }
        info->status = rc;
    }
    return rc;
}

namespace {

int solve_noalloc(const cg_csr *A, const double *b, double *x, double tol, int32_t maxit, void *stream,
                  cg_info *info) {
    if (!A || A->mem != CG_MEM_DEVICE) return CG_EINVAL;
    if (A->n < 0 || A->n > CG_NOALLOC_MAX_N || A->nnz < 0 || A->nnz > (int64_t)INT32_MAX) return CG_EINVAL;
    if (!(tol >= 0.0) || !std::isfinite(tol)) return CG_EINVAL;
    if (A->n == 0) {
        if (info) *info = cg_info{0, CG_OK, 0.0, -1.0, 0.0, 0, 0, -1, 0};
        return CG_OK;
    }
    if (!A->rowptr || !b || !x || b == x || (A->nnz > 0 && (!A->colidx || !A->vals))) return CG_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CG_ECUDA;
    if (!on_device(A->rowptr, dev) || !on_device(b, dev) || !on_device(x, dev) ||
        (A->nnz > 0 && (!on_device(A->colidx, dev) || !on_device(A->vals, dev))))
        return CG_EINVAL;
    unsigned char *scratch = nullptr;
    int grid = 0;
    int rc = noalloc_setup(dev, &scratch, &grid);
    if (rc != CG_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    NoallocArgs args{A->n, A->rowptr, A->colidx, A->vals, b, x, tol, maxit > 0 ? maxit : A->n};
    Params P{};
    P.n = A->n;
    P.r = reinterpret_cast<double *>(scratch + kOffR);
    P.p0 = reinterpret_cast<double *>(scratch + kOffP);
    P.q = reinterpret_cast<double *>(scratch + kOffQ);
    P.partials = reinterpret_cast<double *>(scratch + kOffPartials);
    P.bar = reinterpret_cast<unsigned int *>(scratch + kOffBar);
    P.st = reinterpret_cast<DevStatus *>(scratch + kOffStatus);
    P.tol = tol;
    P.maxit = args.maxit;
    P.phantom = 0;
    P.wait_ns = 5000000000ull;
    int64_t nnz = A->nnz;

    // what must start at zero: the barrier counter and the status block
    cudaError_t e = cudaMemsetAsync(scratch + kOffBar, 0, 256 + 256, st);
    if (e == cudaSuccess) {
        void *kargs[] = {&args, &P, &nnz};
        e = cudaLaunchCooperativeKernel((const void *)cg_noalloc_kernel, dim3(grid), dim3(kThreads), kargs,
                                        (size_t)kNoallocSmem, st);
    }
    DevStatus s{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&s, scratch + kOffStatus, sizeof(DevStatus), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return CG_ECUDA;
    const double bn = std::sqrt(s.bb);
    if (info) {
        *info = cg_info{};
        info->iters = s.iters;
        info->status = s.status;
        info->relres = bn > 0.0 ? std::sqrt(s.rr) / bn : 0.0;
        info->relres_true = -1.0;
        info->kernel_ms = 0.0;
        info->launches = 1;
        info->outer = 0;
        info->reverted_at = -1;
    }
    return s.status;
}

}  // namespace
