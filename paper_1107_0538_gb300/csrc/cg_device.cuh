// Device building blocks of the CG kernels (sm_103a): TMA bulk copies and
// mbarriers, bounded waits, deterministic reductions, the bounded grid
// barrier, and the tiled CSR SpMV that streams the matrix through shared
// memory.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gbcg.h"

namespace gbcg {

// ---------------------------------------------------------------- geometry
// FP64 arithmetic is the scarce resource on GB300 (about 2 FP64 FMA per clock
// per SM, 56x below FP32), so the SpMV gives every row to one thread: exactly
// one FMA per stored entry, no cross-lane reduction adds, no padded slots.
// Each warp streams its own tiles of up to 32 rows through its own shared
// memory stage with TMA bulk copies and its own mbarrier, so warps never
// wait for each other inside the SpMV.
constexpr int kThreads = 512;                  // threads per CTA
constexpr int kWarps = kThreads / 32;
constexpr int kTileRows = 32;                  // rows per warp tile (one per lane)
constexpr int kTileNnz = 1024;                 // stored entries per warp tile
constexpr int kBatch = 9;                      // gathers in flight per thread
constexpr int kValsStage = kTileNnz + 8;       // doubles per stage (alignment slack)
constexpr int kColsStage = kTileNnz + 8;       // int32 per stage
constexpr int kRptrStage = kTileRows + 8;      // int32 per stage (row pointers)
constexpr int kStageBytes = kValsStage * 8 + kColsStage * 4 + kRptrStage * 4;
constexpr int kRedSlots = 4;                   // partial sums per CTA per barrier
constexpr int kSmemBytes = kWarps * kStageBytes + kWarps * 8 /*mbarriers*/ +
                           kWarps * kRedSlots * 8 + 64 /*broadcast*/;
static_assert(kStageBytes % 16 == 0, "stage alignment");
static_assert(kTileNnz + 6 <= kColsStage && kTileNnz + 2 <= kValsStage, "stage slack");
static_assert(kTileRows + 1 + 6 <= kRptrStage, "row pointer slack");

// One row tile: rows [r0, r1) holding entries [a, e).
struct TileDesc {
    int32_t r0, r1, a, e;
};

// Device status block read back once per solve.
struct DevStatus {
    int32_t iters;
    int32_t status;
    double rr;        // ||r_k||^2 at exit
    double bb;        // ||b||^2
    double true_rr;   // ||b - A x||^2 (if computed)
    int32_t where;    // diagnostic: which wait timed out (0 = none)
    int32_t pad;
};

// Everything a kernel needs, passed by value.
struct Params {
    int32_t n;
    const int32_t *__restrict__ rowptr;
    const int32_t *__restrict__ colidx;   // padded to a multiple of 4 + slack
    const double *__restrict__ vals;      // padded to a multiple of 2 + slack
    const int4 *__restrict__ tiles;       // ntiles descriptors (TileDesc)
    const int32_t *__restrict__ cta_tile; // gridDim.x + 1 tile boundaries
    const int32_t *__restrict__ cta_row;  // gridDim.x + 1 row boundaries
    const double *__restrict__ dinv;      // Jacobi: 1 / diag(A), else nullptr
    const double *b;
    double *x;
    double *r;
    double *z;          // == r for plain CG
    double *p0;         // search direction p
    double *q;
    double *partials;   // 2 sets x gridDim.x x kRedSlots
    unsigned int *bar;  // grid barrier counter (zeroed before each launch)
    DevStatus *st;
    double tol;
    int32_t maxit;
    int32_t precond;
    int32_t true_res;
    int32_t phantom;
    unsigned long long wait_ns;
    int32_t evict_first;
};

// ------------------------------------------------------------- primitives
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Waits for phase `parity` of an mbarrier; gives up after limit_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  unsigned long long limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > limit_ns) return false;
    }
    return true;
}

// 1-D bulk copy global -> shared through the TMA unit, completing on `bar`.
// Both addresses 16-byte aligned, bytes a positive multiple of 16.
__device__ __forceinline__ void tma_load_1d(void *dst_smem, const void *src_gmem, uint32_t bytes,
                                            uint64_t *bar, bool evict_first) {
    if (evict_first) {
        uint64_t policy;
        asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(policy));
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
            " [%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst_smem)),
            "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
            : "memory");
    } else {
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes"
            " [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst_smem)),
            "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
            : "memory");
    }
}

__device__ __forceinline__ void red_release_add(unsigned int *addr, unsigned int v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(addr), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int *addr) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(addr) : "memory");
    return v;
}

__device__ __forceinline__ double warp_sum(double v) {
    // xor butterfly: every lane ends with the same bits (a+b == b+a)
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    return v;
}

// Records the first error of a solve (later ones are dropped).
__device__ __forceinline__ void set_error(DevStatus *st, int code, int where) {
    if (atomicCAS(&st->status, 0, code) == 0) st->where = where;
}

// ------------------------------------------------------- shared memory map
struct Smem {
    unsigned char *stage;   // kWarps x kStageBytes (one stage per warp)
    uint64_t *mbar;         // kWarps
    double *red;            // kWarps x kRedSlots
    double *bcast;          // 4 doubles
    int *flag;              // 1 int
    __device__ __forceinline__ double *vals(int s) const {
        return reinterpret_cast<double *>(stage + s * kStageBytes);
    }
    __device__ __forceinline__ int32_t *cols(int s) const {
        return reinterpret_cast<int32_t *>(stage + s * kStageBytes + kValsStage * 8);
    }
    __device__ __forceinline__ int32_t *rptr(int s) const {
        return reinterpret_cast<int32_t *>(stage + s * kStageBytes + kValsStage * 8 + kColsStage * 4);
    }
};

__device__ __forceinline__ Smem carve_smem(unsigned char *base) {
    Smem S;
    S.stage = base;
    S.mbar = reinterpret_cast<uint64_t *>(base + kWarps * kStageBytes);
    S.red = reinterpret_cast<double *>(base + kWarps * kStageBytes + kWarps * 8);
    S.bcast = S.red + kWarps * kRedSlots;
    S.flag = reinterpret_cast<int *>(S.bcast + 4);
    return S;
}

__device__ __forceinline__ void init_pipeline(const Smem &S) {
    if (threadIdx.x == 0) {
        for (int s = 0; s < kWarps; ++s) mbar_init(&S.mbar[s], 1);
        mbar_init_fence();
    }
    __syncthreads();
}

// ---------------------------------------------- deterministic reductions
// Sums NV per-thread values over the CTA in a fixed order; thread 0 returns
// the totals (other threads get unspecified values).
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], const Smem &S) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = warp_sum(v[j]);
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) S.red[warp * kRedSlots + j] = v[j];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            double t = lane < kWarps ? S.red[lane * kRedSlots + j] : 0.0;
            v[j] = warp_sum(t);
        }
    }
    __syncthreads();
}

// Writes this CTA's partial sums (held by thread 0) for barrier set `set`.
template <int NV>
__device__ __forceinline__ void publish_partials(const Params &P, int set, const double (&v)[NV]) {
    if (threadIdx.x == 0) {
        double *dst = P.partials + ((size_t)set * gridDim.x + blockIdx.x) * kRedSlots;
#pragma unroll
        for (int j = 0; j < NV; ++j) dst[j] = v[j];
    }
}

// Sums the partials of every CTA for barrier set `set` in a fixed order; all
// threads of all CTAs obtain bitwise-identical totals.
template <int NV>
__device__ __forceinline__ void grid_totals(const Params &P, int set, const Smem &S,
                                            double (&out)[NV]) {
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {
        const double *src = P.partials + (size_t)set * gridDim.x * kRedSlots;
        const int G = (int)gridDim.x;
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            double s = 0.0;
            for (int m0 = 0; m0 < G; m0 += 32 * 8) {
                double v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int m = m0 + lane + 32 * u;
                    v[u] = m < G ? __ldcg(src + (size_t)m * kRedSlots + j) : 0.0;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) s += v[u];
            }
            s = warp_sum(s);
            if (lane == 0) S.bcast[j] = s;
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NV; ++j) out[j] = S.bcast[j];
}

// Grid-wide barrier on a monotonically increasing counter: barrier number
// `epoch` (1, 2, ...) completes when the counter reaches
// epoch * (gridDim.x + phantom).  Release/acquire at GPU scope make every
// write before the barrier visible to every read after it.  The wait is
// bounded by P.wait_ns; on timeout the error is recorded and false returned
// by every thread of the CTA.
__device__ __forceinline__ bool grid_barrier(const Params &P, unsigned int &epoch, const Smem &S) {
    __syncthreads();
    ++epoch;
    if (threadIdx.x == 0) {
        const unsigned int target = epoch * (gridDim.x + (unsigned)P.phantom);
        red_release_add(P.bar, 1u);
        int ok = 1;
        if (ld_acquire(P.bar) < target) {
            const unsigned long long t0 = global_ns();
            unsigned int spins = 0;
            while (ld_acquire(P.bar) < target) {
                if ((++spins & 63u) == 0 && global_ns() - t0 > P.wait_ns) {
                    ok = 0;
                    break;
                }
            }
        }
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        if (!ok) set_error(P.st, CG_ETIMEOUT, 1);
        S.flag[0] = ok;
    }
    __syncthreads();
    return S.flag[0] != 0;
}

// ------------------------------------------------------------ tiled SpMV
// Sources of the vector the SpMV multiplies.
struct SrcVec {   // v_j = x_j
    const double *x;
    __device__ __forceinline__ double operator()(int j) const { return x[j]; }
};

__device__ __forceinline__ TileDesc load_desc(const Params &P, int t) {
    const int4 d = __ldg(P.tiles + t);
    return TileDesc{d.x, d.y, d.z, d.w};
}

// Per-warp TMA pipeline.  Warp w of a CTA owns the CTA's tiles w, w + kWarps,
// w + 2 kWarps, ... (m of them per pass).  Its running count c over all
// passes maps to local tile w + kWarps (c mod m); the warp's single stage
// completes mbarrier phase c mod 2 for count c.  The matrix never changes, so
// after consuming its last tile of a pass the warp already issues its first
// tile of the next pass: that copy overlaps the vector phase and the grid
// barriers.
struct Pipe {
    uint32_t consumed = 0;
    uint32_t issued = 0;
};

// Issues the TMA copies of tile t into this warp's stage (lane 0 only):
// values, column indices and the row pointers rowptr[r0 .. r1].
__device__ __forceinline__ void issue_tile(const Params &P, const Smem &S, int t, int w) {
    const TileDesc d = load_desc(P, t);
    if (d.e - d.a > kTileNnz) {  // long row: read straight from global memory
        mbar_arrive(&S.mbar[w]);
        return;
    }
    const int va = d.a & ~1, ve = (d.e + 1) & ~1;              // 16-byte aligned ranges
    const int ca = d.a & ~3, ce = (d.e + 3) & ~3;
    const int ra = d.r0 & ~3, re = (d.r1 + 1 + 3) & ~3;
    const uint32_t vbytes = (uint32_t)(ve - va) * 8u, cbytes = (uint32_t)(ce - ca) * 4u;
    const uint32_t rbytes = (uint32_t)(re - ra) * 4u;
    mbar_arrive_expect_tx(&S.mbar[w], vbytes + cbytes + rbytes);
    if (vbytes) {
        tma_load_1d(S.vals(w), P.vals + va, vbytes, &S.mbar[w], P.evict_first != 0);
        tma_load_1d(S.cols(w), P.colidx + ca, cbytes, &S.mbar[w], P.evict_first != 0);
    }
    tma_load_1d(S.rptr(w), P.rowptr + ra, rbytes, &S.mbar[w], false);
}

// Row sums of this CTA's rows: epi.row(i, sum_k vals[k] * src(colidx[k])) is
// called once per row by one thread.  `limit` caps the running count of
// issued tiles per warp (the plain SpMV kernel allows one pass; the solver
// lets each warp run one tile ahead and drains at the end).  Returns false in
// every thread of the CTA if a TMA wait ran out (the error is recorded).
template <class Src, class Epi>
__device__ __forceinline__ bool spmv_tiles(const Params &P, const Smem &S, Pipe &pp,
                                           const Src &src, Epi &epi, bool one_pass = false) {
    const int t0 = P.cta_tile[blockIdx.x], t1 = P.cta_tile[blockIdx.x + 1];
    const int nt = t1 - t0;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m = nt > w ? (nt - w + kWarps - 1) / kWarps : 0;   // this warp's tiles per pass
    bool failed = false;
    if (m > 0) {
        const uint32_t limit = one_pass ? (uint32_t)m : 0xffffffffu;
        if (pp.issued == pp.consumed && pp.issued < limit) {   // nothing in flight yet
            if (lane == 0) issue_tile(P, S, t0 + w, w);
            ++pp.issued;
        }
        for (int j = 0; j < m; ++j) {
            const uint32_t c = pp.consumed;
            const int t = t0 + w + kWarps * (int)(c % (uint32_t)m);
            const TileDesc d = load_desc(P, t);
            const bool got = mbar_wait_bounded(&S.mbar[w], c & 1u, P.wait_ns);
            if (__any_sync(0xffffffffu, !got)) {
                failed = true;
                break;
            }
            if (d.e - d.a > kTileNnz) {
                // one long row: the warp reduces it straight from global memory
                double part = 0.0;
                for (int k = d.a + lane; k < d.e; k += 32) part = fma(P.vals[k], src(P.colidx[k]), part);
                part = warp_sum(part);
                if (lane == 0) epi.row(d.r0, part);
            } else {
                const double *vs = S.vals(w) - (d.a & ~1);
                const int32_t *cs = S.cols(w) - (d.a & ~3);
                const int32_t *rs = S.rptr(w) - (d.r0 & ~3);
                const int row = d.r0 + lane;
                if (row < d.r1) {
                    const int k0 = rs[row], k1 = rs[row + 1];
                    // two interleaved accumulators halve the dependent FMA chain
                    double s0 = 0.0, s1 = 0.0;
                    for (int kb = k0; kb < k1; kb += kBatch) {
                        double v[kBatch], xv[kBatch];
#pragma unroll
                        for (int u = 0; u < kBatch; ++u) {
                            const int k = kb + u;
                            const int col = k < k1 ? cs[k] : -1;
                            v[u] = k < k1 ? vs[k] : 0.0;
                            xv[u] = col >= 0 ? src(col) : 0.0;
                        }
#pragma unroll
                        for (int u = 0; u < kBatch; ++u) {
                            if (kb + u < k1) {
                                if (u & 1) s1 = fma(v[u], xv[u], s1);
                                else s0 = fma(v[u], xv[u], s0);
                            }
                        }
                    }
                    epi.row(row, s0 + s1);
                }
            }
            __syncwarp();  // every lane is done with the stage
            ++pp.consumed;
            if (pp.issued < limit) {
                if (lane == 0) issue_tile(P, S, t0 + w + kWarps * (int)(pp.issued % (uint32_t)m), w);
                ++pp.issued;
            }
        }
    }
    if (__syncthreads_or(failed)) {
        if (threadIdx.x == 0) set_error(P.st, CG_ETIMEOUT, 2);
        return false;
    }
    return true;
}

// Waits (bounded) for every tile still in flight, so that no TMA copy
// targets shared memory after the CTA exits.
__device__ __forceinline__ void drain(const Params &P, const Smem &S, Pipe &pp) {
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        for (uint32_t c = pp.consumed; c < pp.issued; ++c) {
            if (!mbar_wait_bounded(&S.mbar[w], c & 1u, P.wait_ns)) {
                set_error(P.st, CG_ETIMEOUT, 3);
                break;
            }
        }
    }
    pp.consumed = pp.issued;
    __syncthreads();
}

}  // namespace gbcg
