// Device building blocks of the CG kernels (sm_103a): TMA bulk copies and
// mbarriers, bounded waits, deterministic reductions, the bounded grid
// barrier, and the tiled CSR SpMV that streams the matrix through shared
// memory.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "gbcg.h"
#include "check.cuh"
#include "layout.h"

namespace gbcg {

// Device status block read back once per solve.
struct DevStatus {
    int32_t iters;
    int32_t status;
    double rr;        // ||r_k||^2 at exit
    double bb;        // ||b||^2
    double true_rr;   // ||b - A x||^2 (if computed)
    int32_t where;    // diagnostic: which wait timed out (0 = none)
    int32_t outer;    // refinement steps (mixed precision)
};

// Everything a kernel needs, passed by value.
struct Params {
    int32_t n;
    const int32_t *__restrict__ rowptr;
    const int32_t *__restrict__ colidx;   // padded to a multiple of 4 + slack
    const double *__restrict__ vals;      // padded to a multiple of 2 + slack
    const float *__restrict__ vals32;     // inner values, FP32 (mixed precision)
    const __nv_bfloat16 *__restrict__ vals16;  // inner values, BF16 (mixed precision)
    const float *__restrict__ diag_lo;    // inner diagonal (FP32, row-sum compensated)
    const float *__restrict__ dinv32;     // 1 / diag_lo (inner Jacobi)
    float *r32;         // inner residual
    float *z32;         // inner preconditioned residual (== r32 without Jacobi)
    float *p32;         // vector the inner SpMV gathers: z (padded, 16-byte aligned: window source)
    float *pd32;        // inner direction p
    float *q32;         // A_lo p
    float *d32;         // inner correction
    double inner_tol;
    int32_t max_outer;
    int32_t max_inner;
    const int4 *__restrict__ tiles;       // 2 x ntiles int4 (TileDesc)
    const uint16_t *__restrict__ lcol;    // local column of each entry (windowed tiles)
    const int4 *__restrict__ segs;        // window segments: {first column (even), window offset,
                                          //  doubles copied by TMA, tail column or -1}
    const int32_t *__restrict__ cta_tile; // gridDim.x + 1 tile boundaries
    const int32_t *__restrict__ cta_row;  // gridDim.x + 1 row boundaries
    const double *__restrict__ dinv;      // Jacobi: 1 / diag(A), else nullptr
    const double *b;
    double *x;
    double *r;
    double *z;          // == r for plain CG
    double *p0;         // vector the SpMV gathers (padded, 16-byte aligned): z (FP64 CG), p (IR inner)
    double *pd;         // search direction p of the FP64 CG in memory mode (own rows)
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
    double *red;            // kThreads doubles: block-sum transpose
    double *bcast;          // 8 doubles: scalars broadcast by thread 0
    int *ctl;               // 16 ints: decisions broadcast by thread 0
    __device__ __forceinline__ unsigned char *base(int s) const { return stage + s * kStageBytes; }
    template <class VT, class XT>
    __device__ __forceinline__ VT *vals(int s) const {
        return reinterpret_cast<VT *>(base(s) + StageLayout<sizeof(VT), sizeof(XT)>::vals_off);
    }
    template <class VT, class XT>
    __device__ __forceinline__ int32_t *cols(int s) const {
        return reinterpret_cast<int32_t *>(base(s) + StageLayout<sizeof(VT), sizeof(XT)>::cols_off);
    }
    template <class VT, class XT>
    __device__ __forceinline__ int32_t *rptr(int s) const {
        return reinterpret_cast<int32_t *>(base(s) + StageLayout<sizeof(VT), sizeof(XT)>::rptr_off);
    }
    template <class VT, class XT>
    __device__ __forceinline__ XT *win(int s) const {
        return reinterpret_cast<XT *>(base(s) + StageLayout<sizeof(VT), sizeof(XT)>::win_off);
    }
};

__device__ __forceinline__ Smem carve_smem(unsigned char *base) {
    Smem S;
    S.stage = base;
    S.mbar = reinterpret_cast<uint64_t *>(base + kWarps * kStageBytes);
    S.red = reinterpret_cast<double *>(base + kWarps * kStageBytes + kWarps * 8);
    S.bcast = S.red + kThreads;
    S.ctl = reinterpret_cast<int *>(S.bcast + 8);
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
// A warp-wide FP64 instruction costs the same FP64-pipe time however many of
// its lanes are active, so the sums below keep FP64 work to one warp: every
// thread parks its value in shared memory (no FP64 op) and warp 0 adds the
// kThreads values (kThreads / 32 adds per lane in a fixed order, then a
// 5-level butterfly).  Thread 0 returns the totals; the order is the same in
// every CTA and every run.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], const Smem &S) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        S.red[threadIdx.x] = v[j];
        __syncthreads();
        if (threadIdx.x < 32) {
            double t = S.red[lane];
#pragma unroll
            for (int m = 1; m < kWarps; ++m) t += S.red[lane + 32 * m];
            v[j] = warp_sum(t);
        }
        __syncthreads();
    }
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

// Sums the partials of every CTA for barrier set `set` in a fixed order
// (warp 0 only); thread 0 gets the totals, bitwise identical in every CTA.
template <int NV>
__device__ __forceinline__ void grid_totals(const Params &P, int set, double (&out)[NV]) {
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
            out[j] = warp_sum(s);
        }
    }
}

// IEEE finiteness from the exponent bits (integer ops, not the FP64 pipe).
__device__ __forceinline__ bool finite_bits(double v) {
    return ((__double_as_longlong(v) >> 52) & 0x7ff) != 0x7ff;
}

// Grid-wide barrier on a monotonically increasing counter: barrier number
// `epoch` (1, 2, ...) completes when the counter reaches
// epoch * (gridDim.x + phantom).  Release/acquire at GPU scope make every
// write before the barrier visible to every read after it.  The wait is
// bounded by P.wait_ns; on timeout the error is recorded and false returned
// by every thread of the CTA.
// The barrier in two halves, for a CTA that works while it waits: every
// thread calls grid_arrive (after the writes the barrier publishes), thread 0
// alone calls grid_wait (the bounded wait; 1 = passed), and a __syncthreads
// after it releases the CTA.
// FENCE adds a fence.acq_rel.gpu after the wait.  Without it the ordering
// comes from the poll that sees the barrier complete, an ld.acquire.gpu,
// carried to the rest of the CTA by the __syncthreads that follows: under
// the PTX memory model every generic-proxy read after the barrier (L1-cached
// loads included) then sees every write released before it, and a GB300
// saves about 0.4 us per barrier.  Kernels that read, with TMA (the async
// proxy), data that other CTAs wrote keep the fence.
__device__ __forceinline__ void grid_arrive(const Params &P, unsigned int &epoch) {
    __syncthreads();
    ++epoch;
    if (threadIdx.x == 0) red_release_add(P.bar, 1u);
}

template <bool FENCE = true>
__device__ __forceinline__ int grid_wait(const Params &P, unsigned int epoch) {
    const unsigned int target = epoch * (gridDim.x + (unsigned)P.phantom);
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
    if constexpr (FENCE) asm volatile("fence.acq_rel.gpu;" ::: "memory");
    if (!ok) set_error(P.st, CG_ETIMEOUT, 1);
    return ok;
}

template <bool FENCE = true>
__device__ __forceinline__ bool grid_barrier(const Params &P, unsigned int &epoch, const Smem &S) {
    grid_arrive(P, epoch);
    if (threadIdx.x == 0) S.ctl[15] = grid_wait<FENCE>(P, epoch);
    __syncthreads();
    return S.ctl[15] != 0;
}

// ------------------------------------------------------------ tiled SpMV
__device__ __forceinline__ TileDesc load_desc(const Params &P, int t) {
    const int4 d0 = __ldg(P.tiles + 2 * t), d1 = __ldg(P.tiles + 2 * t + 1);
    return TileDesc{d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
}

// Per-warp TMA pipeline.  Warp w of a CTA owns the CTA's tiles w, w + kWarps,
// w + 2 kWarps, ... (m of them per pass).  Its running count c over all
// passes maps to local tile w + kWarps (c mod m) and completes phase c mod 2
// of the warp's mbarrier.  The matrix part of a tile (values, columns, row
// pointers) never changes, so the warp issues it one tile ahead, across
// passes too: the first tile of the next SpMV loads while the vector phases
// and grid barriers run.  The x-window part can only be issued once the
// multiplied vector is final, i.e. inside the pass that uses it; the
// mbarrier expects both parts from the start.
struct Pipe {
    uint32_t consumed = 0;
    uint32_t issued = 0;      // tiles whose matrix part is issued
    uint32_t win_issued = 0;  // tiles whose window part is issued
};

// Conversions of stored values to the accumulation type.
__device__ __forceinline__ double to_acc(double v, double) { return v; }
__device__ __forceinline__ float to_acc(float v, float) { return v; }
__device__ __forceinline__ float to_acc(__nv_bfloat16 v, float) { return __bfloat162float(v); }

// Matrix part of a tile into stage s (lane 0): values (type VT), column
// indices, row pointers; the mbarrier also expects the tile's window of XT
// elements.
template <class VT, class XT>
__device__ __forceinline__ void issue_matrix(const Params &P, const Smem &S, const TileDesc &d, int s,
                                             const VT *vals) {
    if (d.kind == kTileLong) {
        mbar_arrive(&S.mbar[s]);
        return;
    }
    constexpr int epb = 16 / (int)sizeof(VT);        // values per 16 bytes
    const int va = d.a & ~(epb - 1), ve = (d.e + epb - 1) & ~(epb - 1);
    const int ra = d.r0 & ~3, re = (d.r1 + 1 + 3) & ~3;
    const uint32_t vbytes = (uint32_t)(ve - va) * (uint32_t)sizeof(VT), rbytes = (uint32_t)(re - ra) * 4u;
    uint32_t cbytes;
    const void *csrc;
    if (d.kind == kTileWindow) {
        const int ca = d.a & ~7, ce = (d.e + 7) & ~7;
        cbytes = (uint32_t)(ce - ca) * 2u;
        csrc = P.lcol + ca;
    } else {
        const int ca = d.a & ~3, ce = (d.e + 3) & ~3;
        cbytes = (uint32_t)(ce - ca) * 4u;
        csrc = P.colidx + ca;
    }
    // window bytes the TMA will deliver (tail columns are stored by threads)
    const uint32_t wbytes = (uint32_t)d.wtx * (uint32_t)sizeof(XT);
    mbar_arrive_expect_tx(&S.mbar[s], (d.e > d.a ? vbytes + cbytes : 0u) + rbytes + wbytes);
    if (d.e > d.a) {
        tma_load_1d(S.vals<VT, XT>(s), vals + va, vbytes, &S.mbar[s], P.evict_first != 0);
        tma_load_1d(S.cols<VT, XT>(s), csrc, cbytes, &S.mbar[s], P.evict_first != 0);
    }
    tma_load_1d(S.rptr<VT, XT>(s), P.rowptr + ra, rbytes, &S.mbar[s], false);
}

// Window part of a windowed tile into stage s: lane l copies segment l of
// the vector x (16-byte aligned).
template <class VT, class XT>
__device__ __forceinline__ void issue_window(const Params &P, const Smem &S, const TileDesc &d, int s,
                                             const XT *x) {
    const int lane = threadIdx.x & 31;
    if (d.kind != kTileWindow || lane >= d.nseg) return;
    const int4 sg = __ldg(P.segs + d.seg0 + lane);
    if (sg.z > 0)
        tma_load_1d(S.win<VT, XT>(s) + sg.y, x + sg.x, (uint32_t)sg.z * (uint32_t)sizeof(XT), &S.mbar[s], false);
}

// A segment running past the vector's end stops at column n & ~3; its lane
// stores the 1 to 3 columns after that into the window slots that follow.
template <class VT, class XT>
__device__ __forceinline__ void store_tail(const Params &P, const Smem &S, const TileDesc &d, int s,
                                           const XT *x) {
    const int lane = threadIdx.x & 31;
    if (d.kind != kTileWindow || lane >= d.nseg) return;
    const int4 sg = __ldg(P.segs + d.seg0 + lane);
    if (sg.w >= 0) {
        XT *win = S.win<VT, XT>(s);
        for (int c = sg.w; c < P.n; ++c) win[sg.y + sg.z + (c - sg.w)] = x[c];
    }
}

template <class VT, class XT>
__device__ __forceinline__ void issue_next(const Params &P, const Smem &S, Pipe &pp, int t0, int m,
                                           uint32_t limit, uint32_t pass_end, const VT *vals, const XT *x) {
    const int w = threadIdx.x >> 5;
    if (pp.issued < pp.consumed + 1 && pp.issued < limit) {
        const TileDesc d = load_desc(P, t0 + w + kWarps * (int)(pp.issued % (uint32_t)m));
        // order this warp's generic shared-memory writes to the stage (tail
        // columns) before the async-proxy copies that will overwrite it
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if ((threadIdx.x & 31) == 0) issue_matrix<VT, XT>(P, S, d, w, vals);
        __syncwarp();
        if (pp.issued < pass_end) {  // same pass: the vector is final, load the window now
            issue_window<VT, XT>(P, S, d, w, x);
            ++pp.win_issued;
        }
        ++pp.issued;
    }
}

// Sum over one row: exactly one FMA per stored entry, the loads of a batch
// issued before its first FMA, two interleaved accumulators.
template <class AT, class VT, class Col, class Val>
__device__ __forceinline__ AT row_sum(int k0, int k1, const Col &col_of, const Val &val_of, const VT *vs) {
    AT s0 = AT(0), s1 = AT(0);
    for (int kb = k0; kb < k1; kb += kBatch) {
        AT v[kBatch], xv[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int k = min(kb + u, k1 - 1);  // clamped: every load is in range
            v[u] = to_acc(vs[k], AT(0));
            xv[u] = val_of(col_of(k));
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            if (kb + u < k1) {
                if (u & 1) s1 = fma(v[u], xv[u], s1);
                else s0 = fma(v[u], xv[u], s0);
            }
        }
    }
    return s0 + s1;
}

// Epilogues that read vector entries of their row may define prefetch(i):
// it is called with the lane's row before the wait for the tile's stage, so
// those loads overlap the wait and the row sum instead of following it.
template <class E>
__device__ __forceinline__ auto maybe_prefetch(E &e, int i, int) -> decltype(e.prefetch(i), void()) {
    e.prefetch(i);
}
template <class E>
__device__ __forceinline__ void maybe_prefetch(E &, int, long) {}

// One tile of a warp: waits for its stage, forms the row sums and calls
// epi.row(i, sum, j) for each row i of the tile (lane l gets row r0 + l; j is
// the warp's local tile number in the pass).  Returns false if the wait ran
// out.
template <class VT, class XT, class AT, class Epi>
__device__ __forceinline__ bool warp_tile(const Params &P, const Smem &S, Pipe &pp, int t0, int m,
                                          uint32_t limit, uint32_t pass_end, const VT *vals, const XT *x,
                                          Epi &epi, int j) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t c = pp.consumed;
    const TileDesc d = load_desc(P, t0 + w + kWarps * (int)(c % (uint32_t)m));
    store_tail<VT, XT>(P, S, d, w, x);  // nobody reads the stage before the wait below
    {
        const int prow = d.kind == kTileLong ? d.r0 : d.r0 + lane;
        if (prow < d.r1) maybe_prefetch(epi, prow, 0);
    }
    const bool got = mbar_wait_bounded(&S.mbar[w], c & 1u, P.wait_ns);
    if (__any_sync(0xffffffffu, !got)) return false;
    __syncwarp();
    if (d.kind == kTileLong) {
        // one long row: the warp reduces it straight from global memory
        AT part = AT(0);
        for (int k = d.a + lane; k < d.e; k += 32)
            part = fma(to_acc(vals[k], AT(0)), AT(x[bchk(P.colidx[k], P.n)]), part);
#pragma unroll
        for (int mm = 16; mm >= 1; mm >>= 1) part += __shfl_xor_sync(0xffffffffu, part, mm);
        if (lane == 0) epi.row(d.r0, part, j);
    } else {
        const VT *vs = S.vals<VT, XT>(w) - (d.a & ~(16 / (int)sizeof(VT) - 1));
        const int32_t *rs = S.rptr<VT, XT>(w) - (d.r0 & ~3);
        const int row = d.r0 + lane;
        if (row < d.r1) {
            int k0 = rs[row], k1 = rs[row + 1];
            bchk_range(k0, k1, d.a, d.e);
            AT sum = AT(0);
            if (k1 > k0) {
                if (d.kind == kTileWindow) {
                    const uint16_t *lc = reinterpret_cast<const uint16_t *>(S.cols<VT, XT>(w)) - (d.a & ~7);
                    const XT *win = S.win<VT, XT>(w);
                    sum = row_sum<AT>(k0, k1, [&](int k) { return (int)lc[k]; },
                                      [&](int c2) { return AT(win[bchk(c2, kWinMax)]); }, vs);
                } else {
                    const int32_t *cs = S.cols<VT, XT>(w) - (d.a & ~3);
                    sum = row_sum<AT>(k0, k1, [&](int k) { return cs[k]; },
                                      [&](int c2) { return AT(x[bchk(c2, P.n)]); }, vs);
                }
            }
            epi.row(row, sum, j);
        }
    }
    __syncwarp();  // every lane is done with the stage
    ++pp.consumed;
    issue_next<VT, XT>(P, S, pp, t0, m, limit, pass_end, vals, x);
    return true;
}

// Row sums of this CTA's rows: epi.row(i, sum_k vals[k] * x[colidx[k]], j)
// is called once per row by the thread that owns it; VT is the stored value
// type, XT the vector element type (x 16-byte aligned), AT the accumulation
// type.  RPT > 0 unrolls the warp's tile loop (at most RPT tiles per warp)
// so that j is a compile-time index into register-resident row state;
// RPT = 0 loops at run time.  `one_pass` stops the pipeline at the end of
// the pass; otherwise the next pass's first tile is left in flight (matrix
// part only, same value type).  Returns false in every thread of the CTA if
// a TMA wait ran out (the error is recorded).
template <int RPT, class VT, class XT, class AT, class Epi>
__device__ __forceinline__ bool spmv_tiles(const Params &P, const Smem &S, Pipe &pp, const VT *vals,
                                           const XT *x, Epi &epi, bool one_pass = false) {
    const int t0 = P.cta_tile[blockIdx.x], t1 = P.cta_tile[blockIdx.x + 1];
    const int nt = t1 - t0;
    const int w = threadIdx.x >> 5;
    const int m = nt > w ? (nt - w + kWarps - 1) / kWarps : 0;   // this warp's tiles per pass
    bool failed = false;
    if (m > 0) {
        const uint32_t pass_end = pp.consumed + (uint32_t)m;
        const uint32_t limit = one_pass ? pass_end : 0xffffffffu;
        // windows of tiles whose matrix part was issued during the last pass
        while (pp.win_issued < pp.issued) {
            const TileDesc d = load_desc(P, t0 + w + kWarps * (int)(pp.win_issued % (uint32_t)m));
            issue_window<VT, XT>(P, S, d, w, x);
            ++pp.win_issued;
        }
        issue_next<VT, XT>(P, S, pp, t0, m, limit, pass_end, vals, x);
        if (RPT > 0) {
#pragma unroll
            for (int j = 0; j < (RPT > 0 ? RPT : 1); ++j) {
                if (j < m && !failed)
                    failed = !warp_tile<VT, XT, AT>(P, S, pp, t0, m, limit, pass_end, vals, x, epi, j);
            }
        } else {
            for (int j = 0; j < m && !failed; ++j)
                failed = !warp_tile<VT, XT, AT>(P, S, pp, t0, m, limit, pass_end, vals, x, epi, j);
        }
    }
    if (__syncthreads_or(failed)) {
        if (threadIdx.x == 0) set_error(P.st, CG_ETIMEOUT, 2);
        return false;
    }
    return true;
}

// Waits (bounded) for every tile still in flight, so that no TMA copy
// targets shared memory after the CTA exits.  A prefetched tile whose window
// was never issued cannot complete its phase, so the window is issued first
// (from any vector: the data is not used).
template <class VT, class XT>
__device__ __forceinline__ void drain(const Params &P, const Smem &S, Pipe &pp, const XT *any_x) {
    const int w = threadIdx.x >> 5;
    const int t0 = P.cta_tile[blockIdx.x], nt = P.cta_tile[blockIdx.x + 1] - t0;
    const int m = nt > w ? (nt - w + kWarps - 1) / kWarps : 0;
    if (m > 0) {
        while (pp.win_issued < pp.issued) {
            const TileDesc d = load_desc(P, t0 + w + kWarps * (int)(pp.win_issued % (uint32_t)m));
            issue_window<VT, XT>(P, S, d, w, any_x);
            ++pp.win_issued;
        }
        if ((threadIdx.x & 31) == 0) {
            for (uint32_t c = pp.consumed; c < pp.issued; ++c) {
                if (!mbar_wait_bounded(&S.mbar[w], c & 1u, P.wait_ns)) {
                    set_error(P.st, CG_ETIMEOUT, 3);
                    break;
                }
            }
        }
    }
    pp.consumed = pp.issued;
    __syncthreads();
}

}  // namespace gbcg
