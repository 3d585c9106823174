// Batched solves: many independent SPD systems, each with up to four
// right-hand sides, in one persistent cooperative launch.
//
// The systems are laid out as one block-diagonal CSR matrix whose row tiles
// never cross a system; every (system, right-hand side) pair runs its own
// mixed-precision iterative refinement (FP64 outer residual and solution
// with the FP64 matrix, FP32 inner CG on the rounded matrix, optional
// Jacobi), all pairs in lockstep through the same grid barriers:
//
//   outer step   r = b - A x per right-hand side (FP64 SpMV), stop test on
//                ||r|| <= tol ||b||, inner start r_in = z = p = M^-1 r, d = 0
//   inner loop   q = A_lo p for the four right-hand sides at once (the matrix
//                tile is streamed once; the x-window holds float4), then
//                d, r_in, z and p updates; each pair leaves the inner loop
//                when its residual fell by inner_tol
//   x += d       for the pairs that ran an inner solve
//
// Reductions are per pair: each warp accumulates its rows' contributions per
// (CTA, system) segment and flushes them to memory; per segment the 16 warp
// sums are added in a fixed order, and after the grid barrier every CTA adds
// each system's segments in a fixed order, so every CTA takes the same
// decisions for every pair (results are bitwise reproducible).  Tiles of
// systems whose pairs are all done are skipped, so the work shrinks as
// systems converge.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "cg_device.cuh"
#include "gbcg.h"
#include "handle.h"
#include "lowprec.h"
#include "plan.h"

using namespace gbcg;

namespace {

constexpr int kRhs = 4;        // right-hand sides streamed together
constexpr int kSlots = 12;     // partial sums per segment and pass
constexpr int kMaxSegPerCta = 64;

// Per-pair solver state; every CTA keeps its own identical copy.
struct PairState {
    double rho;        // inner r.z
    double bnorm;      // ||b||
    double relres;     // last outer ||b - A x|| / ||b||
    double target2;    // (inner_tol ||r_outer||)^2
    float alpha, beta;
    int32_t flags;     // bit 0: outer active, bit 1: inner active, bit 2: ran inner this step
    int32_t iters, outer, status;
};
constexpr int kOuterActive = 1, kInnerActive = 2, kRanInner = 4;

struct BatchParams {
    Params P;                    // shared fields: tiles, segs, lcol, rowptr, colidx, vals,
                                 // vals32/vals16, diag_lo, dinv32, bar, wait_ns, precond, n
    const int32_t *tile_sys;     // system of each tile
    const int32_t *cta_sys0;     // first system of each CTA
    const int32_t *cta_nsys;
    const int32_t *cta_seg0;     // first segment of each CTA (ctas + 1)
    const int32_t *sys_seg0;     // first segment of each system (nsys + 1)
    int32_t nsys, nrhs, nseg;
    int32_t lanes_per_row;       // SpMM rows per warp step: 32 / lanes_per_row (1, 2 or 4 lanes per row)
    double tol, inner_tol;
    int32_t maxit, max_outer, max_inner;
    const double *B;             // caller's right-hand sides, column r at B + r * n
    double *xw;                  // working x, column r at xw + r * xstride (16-byte aligned)
    int32_t xstride;
    float4 *r32, *z32, *p32, *q32, *d32;   // inner vectors, the four right-hand sides interleaved
                                           // (p32: the vector the SpMM gathers, z)
    float4 *pd32;                          // inner directions
    double *wpart;               // ctas x warps x kMaxSegPerCta x kSlots: warp partial sums
    double *segpart;             // 2 x nseg x kSlots
    PairState *state;            // ctas x nsys x kRhs
    cg_batch_result *results;    // nsys x kRhs
    // balanced inner layout (the active tiles split evenly over the CTAs)
    const int32_t *sys_tile0;    // first tile of each system (nsys + 1)
    int32_t *bal;                // ctas x 2 (nsys + 1): per CTA, active-tile and active-system prefixes
    int4 *sinf;                  // ctas x nsys: per CTA, each active system's first and last piece, its
                                 // segment in the first piece (x, y, z) and whether some piece is empty (w)
    double *segdyn;              // 2 x ctas x kMaxSegPerCta x kSlots: per-piece segment sums
    int32_t balance;             // 1: the inner loop may use the balanced layout
};

__device__ __forceinline__ float f4c(const float4 &v, int r) {
    return r == 0 ? v.x : (r == 1 ? v.y : (r == 2 ? v.z : v.w));
}
__device__ __forceinline__ void f4set(float4 &v, int r, float a) {
    if (r == 0) v.x = a;
    else if (r == 1) v.y = a;
    else if (r == 2) v.z = a;
    else v.w = a;
}

// FMA into the accumulation types of the passes.
__device__ __forceinline__ double fma_acc(double v, double x, double a) { return fma(v, x, a); }
__device__ __forceinline__ float4 fma_acc(float v, float4 x, float4 a) {
    return make_float4(fmaf(v, x.x, a.x), fmaf(v, x.y, a.y), fmaf(v, x.z, a.z), fmaf(v, x.w, a.w));
}
__device__ __forceinline__ float4 fma_acc(__nv_bfloat16 v, float4 x, float4 a) {
    return fma_acc(__bfloat162float(v), x, a);
}
__device__ __forceinline__ double xor_add(double v, int m) { return v + __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ float4 xor_add(float4 v, int m) {
    return make_float4(v.x + __shfl_xor_sync(0xffffffffu, v.x, m), v.y + __shfl_xor_sync(0xffffffffu, v.y, m),
                       v.z + __shfl_xor_sync(0xffffffffu, v.z, m), v.w + __shfl_xor_sync(0xffffffffu, v.w, m));
}
__device__ __forceinline__ double warp_sum_acc(double v) { return warp_sum(v); }
__device__ __forceinline__ float4 warp_sum_acc(float4 v) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, m);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, m);
        v.z += __shfl_xor_sync(0xffffffffu, v.z, m);
        v.w += __shfl_xor_sync(0xffffffffu, v.w, m);
    }
    return v;
}


// ---------------------------------------------------------------- passes
// One pass over this warp's tiles (tiles w, w + kWarps, ... of the CTA),
// skipping the tiles `active` rejects.  With a matrix (vals != nullptr) each
// active tile is streamed through the warp's stage (one tile of look-ahead)
// and rowfn(tile, row, j_local_seg, sum) is called per row; without one,
// rowfn(tile, row, seg, 0) is called per row.  Each lane keeps kSlots
// accumulators per segment (acc), flushed to wpart when the warp moves to
// another segment and at the end.
template <class T, int NS>
struct WarpAcc {
    T a[NS > 0 ? NS : 1];
    int seg;
};

// Warp-sums the lanes' accumulators of the current segment (in T: FP32 for
// the inner passes, FP64 for the outer residual) and adds them to the warp's
// own row of wpart (zeroed at the start of each reduction).
template <class T, int NS>
__device__ __forceinline__ void flush_acc(const BatchParams &B, WarpAcc<T, NS> &acc) {
    if (NS == 0) return;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *dst = B.wpart + (((size_t)blockIdx.x * kWarps + w) * kMaxSegPerCta + acc.seg) * kSlots;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        T v = acc.a[i];
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
        if (lane == 0) dst[i] += (double)v;
    }
}

template <class T, int NS>
__device__ __forceinline__ void acc_switch(const BatchParams &B, WarpAcc<T, NS> &acc, int seg) {
    if (seg != acc.seg) {
        if (acc.seg >= 0) flush_acc(B, acc);
        acc.seg = seg;
#pragma unroll
        for (int i = 0; i < (NS > 0 ? NS : 1); ++i) acc.a[i] = T(0);
    }
}

// Zeroes this warp's rows of wpart for ns segments.
__device__ __forceinline__ void zero_wpart(const BatchParams &B, int ns) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *row = B.wpart + ((size_t)blockIdx.x * kWarps + w) * kMaxSegPerCta * kSlots;
    for (int i = lane; i < ns * kSlots; i += 32) row[i] = 0.0;
    __syncwarp();
}

// Adds the 16 warp rows of each of this CTA's segments (fixed order) into
// segpart[set], for the first nslots slots.
__device__ __forceinline__ void combine_segments(const BatchParams &B, int set, int nslots) {
    __syncthreads();
    const int ns = B.cta_nsys[blockIdx.x], seg0 = B.cta_seg0[blockIdx.x];
    const double *wp = B.wpart + (size_t)blockIdx.x * kWarps * kMaxSegPerCta * kSlots;
    for (int q = threadIdx.x; q < ns * nslots; q += kThreads) {
        const int j = q / nslots, i = q % nslots;
        double s = 0.0;
        for (int w = 0; w < kWarps; ++w) s += wp[((size_t)w * kMaxSegPerCta + j) * kSlots + i];
        B.segpart[((size_t)set * B.nseg + seg0 + j) * kSlots + i] = s;
    }
}

// Total of one slot for one system: its segments in a fixed order (T = double
// for the FP64 outer residual, float for the FP32 inner solve).
template <class T>
__device__ __forceinline__ T system_total(const BatchParams &B, int set, int sys, int slot) {
    T s = T(0);
    for (int k = B.sys_seg0[sys]; k < B.sys_seg0[sys + 1]; ++k)
        s += (T)__ldcg(B.segpart + ((size_t)set * B.nseg + k) * kSlots + slot);
    return s;
}

// Row functions that read their row's vector entries may define
// prefetch(row): with one lane per row it is called for the lane's row before
// the wait for the tile's stage, so those loads overlap the wait and the sum.
template <class F>
__device__ __forceinline__ auto batch_prefetch(F &f, int i, int) -> decltype(f.prefetch(i), void()) {
    f.prefetch(i);
}
template <class F>
__device__ __forceinline__ void batch_prefetch(F &, int, long) {}

// ------------------------------------------------------------ tile layouts
// Which tiles a warp takes in a pass.  The static layout is the plan's split:
// CTA c owns tiles cta_tile[c] .. cta_tile[c + 1] (balanced over all
// systems); warp w takes tiles w, w + kWarps, ... of them and skips the tiles
// of systems the pass's predicate rejects.  As systems converge, that leaves
// the CTAs holding the slow systems with all the work while the others wait
// at the barriers.  So the inner loop re-splits whenever a system leaves it:
// the tiles of the systems still active, in system order, are numbered
// 0 .. T-1, CTA c takes the piece [floor(c T / G), floor((c + 1) T / G)) and
// its warp w the tiles w, w + kWarps, ... of the piece.  The segments of a
// piece are the active systems it touches, in order (at most kMaxSegPerCta,
// else the static layout is kept).  Every CTA derives the same layout from
// its copy of the pair states, so a system's partial sums are added in the
// same order everywhere and results stay bitwise reproducible.
constexpr int kMaxBalCtas = 320;   // CTAs the layout arrays in shared memory hold
constexpr int kBalHdr = 2 * kWarps;
constexpr int kBalArr = kBalHdr + 8;
static_assert((kBalArr + 3 * kMaxBalCtas) * 4 <= kThreads * 8, "layout arrays fit the block-sum area");

struct Balance {   // the CTA's view of the current layout (shared memory)
    int dyn;       // 1: balanced layout, 0: the plan's static split
    int v0, v1;    // this CTA's piece of the active tiles
    int s0;        // system holding tile v0 (v0 < v1)
    int k0;        // its active rank
    int nloc;      // segments of the piece
    int total;     // T, active tiles
    int pad;
};

template <class Active>
struct StaticTiles {
    const BatchParams *B;
    const Active *active;
    int t, end, s0;
    __device__ __forceinline__ void skip() {
        while (t < end && !(*active)(B->tile_sys[t])) t += kWarps;
    }
    __device__ __forceinline__ void start(int w) {
        t = B->P.cta_tile[blockIdx.x] + w;
        end = B->P.cta_tile[blockIdx.x + 1];
        s0 = B->cta_sys0[blockIdx.x];
        skip();
    }
    __device__ __forceinline__ bool valid() const { return t < end; }
    __device__ __forceinline__ int tile() const { return t; }
    __device__ __forceinline__ int sys() const { return B->tile_sys[t]; }
    __device__ __forceinline__ int seg() const { return B->tile_sys[t] - s0; }
    __device__ __forceinline__ void next() {
        t += kWarps;
        skip();
    }
};
template <class Active>
__device__ __forceinline__ StaticTiles<Active> static_tiles(const BatchParams &B, const Active &a) {
    return StaticTiles<Active>{&B, &a, 0, 0, 0};
}

// This CTA's prefixes: pfx[s] active tiles and rk[s] active systems before
// system s (nsys + 1 entries each).
__device__ __forceinline__ int32_t *bal_pfx(const BatchParams &B) {
    return B.bal + (size_t)blockIdx.x * 2 * (B.nsys + 1);
}

// Tiles v0 + w, v0 + w + kWarps, ... < v1 of the active-tile numbering.
struct BalancedTiles {
    const BatchParams *B;
    const int32_t *pfx, *rk;
    int v, v1, s, k0;
    __device__ __forceinline__ void settle() {
        if (v < v1)
            while (v >= pfx[s + 1]) ++s;
    }
    __device__ __forceinline__ void start(int w) {
        v += w;
        settle();
    }
    __device__ __forceinline__ bool valid() const { return v < v1; }
    __device__ __forceinline__ int tile() const { return B->sys_tile0[bchk(s, B->nsys)] + (v - pfx[s]); }
    __device__ __forceinline__ int sys() const { return s; }
    __device__ __forceinline__ int seg() const { return rk[s] - k0; }
    __device__ __forceinline__ void next() {
        v += kWarps;
        settle();
    }
};
__device__ __forceinline__ BalancedTiles balanced_tiles(const BatchParams &B, const Balance &L) {
    const int32_t *pfx = bal_pfx(B);
    return BalancedTiles{&B, pfx, pfx + B.nsys + 1, L.v0, L.v1, L.s0, L.k0};
}

// The piece holding active tile v: the largest c with floor(c T / G) <= v.
__device__ __forceinline__ int piece_of(int v, int T, int G) {
    return (int)(((long long)(v + 1) * G - 1) / T);
}

// Builds the balanced layout of the systems `active` accepts: this CTA's
// prefixes and per-system pieces (sinf), every piece's first and last active
// rank (bsm) and the CTA's own piece (L).  Every CTA checks every piece, so
// all take the same decision (dyn) and the same layout.  All threads call it;
// it ends with a __syncthreads.
template <class Active>
__device__ void compute_balance(const BatchParams &B, const Active &active, int *bsm) {
    Balance &L = *reinterpret_cast<Balance *>(bsm + kBalHdr);
    int *scan = bsm, *k0c = bsm + kBalArr, *k1c = k0c + kMaxBalCtas, *s0c = k1c + kMaxBalCtas;
    const int ns = B.nsys, G = (int)gridDim.x;
    int32_t *pfx = bal_pfx(B), *rk = pfx + ns + 1;
    const int per = (ns + kThreads - 1) / kThreads;
    const int a = min((int)threadIdx.x * per, ns), b = min(a + per, ns);
    int tiles = 0, cnt = 0;
    for (int s = a; s < b; ++s)
        if (active(s)) {
            tiles += B.sys_tile0[s + 1] - B.sys_tile0[s];
            ++cnt;
        }
    // exclusive scan of (tiles, cnt) in thread order
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int ti = tiles, ci = cnt;
#pragma unroll
    for (int m = 1; m < 32; m <<= 1) {
        const int tu = __shfl_up_sync(0xffffffffu, ti, m), cu = __shfl_up_sync(0xffffffffu, ci, m);
        if (lane >= m) {
            ti += tu;
            ci += cu;
        }
    }
    if (lane == 31) {
        scan[w] = ti;
        scan[kWarps + w] = ci;
    }
    for (int c = threadIdx.x; c < G; c += kThreads) k0c[c] = k1c[c] = s0c[c] = 0;
    __syncthreads();
    int tb = ti - tiles, cb = ci - cnt, T = 0, K = 0;
    for (int j = 0; j < kWarps; ++j) {
        if (j < w) {
            tb += scan[j];
            cb += scan[kWarps + j];
        }
        T += scan[j];
        K += scan[kWarps + j];
    }
    const long long g = G;
    for (int s = a; s < b; ++s) {
        pfx[s] = tb;
        rk[s] = cb;
        if (active(s)) {
            const long long t0 = tb, t1 = tb + (B.sys_tile0[s + 1] - B.sys_tile0[s]);
            // pieces whose first tile floor(c T / G) lies in [t0, t1)
            for (long long c = (t0 * g + T - 1) / T; c < g && c * T / g < t1; ++c) {
                k0c[c] = cb;
                s0c[c] = s;
            }
            // pieces whose last tile floor((c + 1) T / G) - 1 lies in [t0, t1)
            for (long long c = ((t0 + 1) * g + T - 1) / T - 1; c < g && (c + 1) * T / g <= t1; ++c) k1c[c] = cb;
            tb = (int)t1;
            ++cb;
        }
    }
    if (threadIdx.x == 0) {
        pfx[ns] = T;
        rk[ns] = K;
    }
    __syncthreads();
    // each system's pieces: c0 .. c1, its segment j0 in piece c0 (0 in the
    // later ones, which start inside it); with T < G some pieces are empty
    int4 *sinf = B.sinf + (size_t)blockIdx.x * ns;
    for (int s = a; s < b; ++s) {
        const int t0 = pfx[s], t1 = pfx[s + 1];
        int4 v = make_int4(0, -1, 0, 0);
        if (t1 > t0) {
            v.x = piece_of(t0, T, G);
            v.y = piece_of(t1 - 1, T, G);
            v.z = rk[s] - k0c[v.x];
            v.w = T < G;
        }
        sinf[s] = v;
    }
    int over = 0;
    for (int c = threadIdx.x; c < G; c += kThreads) {
        const long long v0 = (long long)c * T / g, v1 = (long long)(c + 1) * T / g;
        if (v1 > v0 && k1c[c] - k0c[c] + 1 > kMaxSegPerCta) over = 1;
    }
    over = __syncthreads_or(over);
    if (threadIdx.x == 0) {
        const int c = blockIdx.x;
        const int v0 = T > 0 ? (int)((long long)c * T / g) : 0, v1 = T > 0 ? (int)((long long)(c + 1) * T / g) : 0;
        const bool mine = v1 > v0;
        L.dyn = (T > 0 && !over) ? 1 : 0;
        L.total = T;
        L.v0 = v0;
        L.v1 = v1;
        L.s0 = mine ? s0c[c] : 0;
        L.k0 = mine ? k0c[c] : 0;
        L.nloc = mine ? k1c[c] - k0c[c] + 1 : 0;
    }
    __syncthreads();
}

// Adds the 16 warp rows of each of this piece's nloc segments (fixed order)
// into segdyn[set][c], for the first nslots slots.
__device__ __forceinline__ void combine_segments_dyn(const BatchParams &B, int set, int nslots, int nloc) {
    __syncthreads();
    const double *wp = B.wpart + (size_t)blockIdx.x * kWarps * kMaxSegPerCta * kSlots;
    double *dst = B.segdyn + ((size_t)set * gridDim.x + blockIdx.x) * kMaxSegPerCta * kSlots;
    for (int q = threadIdx.x; q < nloc * nslots; q += kThreads) {
        const int j = q / nslots, i = q % nslots;
        double s = 0.0;
        for (int w = 0; w < kWarps; ++w) s += wp[((size_t)w * kMaxSegPerCta + j) * kSlots + i];
        dst[(size_t)j * kSlots + i] = s;
    }
}

// Totals of slots sl[0..NS) for one system under the balanced layout: the
// system's segments in the pieces it spans, in piece order (zero for a
// system outside the layout).
template <int NS>
__device__ __forceinline__ void system_totals_dyn(const BatchParams &B, int set, int total, int sys,
                                                  const int (&sl)[NS], float (&out)[NS]) {
    const int4 v = B.sinf[(size_t)blockIdx.x * B.nsys + sys];
    const int G = (int)gridDim.x;
#pragma unroll
    for (int i = 0; i < NS; ++i) out[i] = 0.0f;
    for (int c = v.x; c <= v.y; ++c) {
        // an empty piece (fewer active tiles than CTAs) holds nothing
        if (v.w && c * total / G == (c + 1) * total / G) continue;
        const int j = c == v.x ? bchk(v.z, kMaxSegPerCta) : 0;
        const double *src = B.segdyn + (((size_t)set * G + c) * kMaxSegPerCta + j) * kSlots;
#pragma unroll
        for (int i = 0; i < NS; ++i) out[i] += (float)__ldcg(src + sl[i]);
    }
}

template <class VT, class XT, class AT, class Cur, class RowFn, class Acc>
__device__ __forceinline__ bool batch_pass(const BatchParams &B, const Smem &S, uint32_t &count,
                                           const VT *vals, const XT *x, Cur cur, RowFn &rowfn,
                                           Acc &acc) {
    const Params &P = B.P;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    bool ok = true;
    cur.start(w);
    if (vals == nullptr) {
        // the next tile's descriptor and row loads (prefetch) are issued
        // before the current tile's rows are finished: two tiles in flight
        TileDesc d{};
        if (cur.valid()) {
            d = load_desc(P, cur.tile());
            if (d.r0 + lane < d.r1) batch_prefetch(rowfn, d.r0 + lane, 0);
        }
        while (cur.valid()) {
            Cur nx = cur;
            nx.next();
            TileDesc dn{};
            if (nx.valid()) {
                dn = load_desc(P, nx.tile());
                if (dn.r0 + lane < dn.r1) batch_prefetch(rowfn, dn.r0 + lane, 0);
            }
            acc_switch(B, acc, cur.seg());
            const int row = d.r0 + lane;
            if (row < d.r1) rowfn(cur.sys(), row, AT{}, acc);
            d = dn;
            cur = nx;
        }
    } else {
        // the descriptor loaded to issue a tile's copies is kept for its turn
        TileDesc dc{};
        if (cur.valid()) {
            const TileDesc d = load_desc(P, cur.tile());
            dc = d;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) issue_matrix<VT, XT>(P, S, d, w, vals);
            __syncwarp();
            issue_window<VT, XT>(P, S, d, w, x);
        }
        while (cur.valid()) {
            const TileDesc d = dc;
            const int sys = cur.sys();
            store_tail<VT, XT>(P, S, d, w, x);
            if (B.lanes_per_row == 1 && d.kind != kTileLong && d.r0 + lane < d.r1) batch_prefetch(rowfn, d.r0 + lane, 0);
            const bool got = mbar_wait_bounded(&S.mbar[w], count & 1u, P.wait_ns);
            if (__any_sync(0xffffffffu, !got)) {
                ok = false;
                break;
            }
            __syncwarp();
            acc_switch(B, acc, cur.seg());
            const int row = d.r0 + lane;
            if (d.kind == kTileLong) {
                AT part{};
                for (int k = d.a + lane; k < d.e; k += 32) part = fma_acc(vals[k], x[bchk(P.colidx[k], P.n)], part);
                part = warp_sum_acc(part);
                if (lane == 0) rowfn(sys, d.r0, part, acc);
            } else {
                // the tile's rows in steps of 32 / L rows, L = lanes_per_row
                // lanes per row (lane l takes entries k0 + l mod L, + L, ...;
                // the L partial sums are joined by a butterfly)
                const VT *vs = S.vals<VT, XT>(w) - (d.a & ~(16 / (int)sizeof(VT) - 1));
                const int32_t *rs = S.rptr<VT, XT>(w) - (d.r0 & ~3);
                const int L = B.lanes_per_row, lg = L == 4 ? 2 : (L == 2 ? 1 : 0);
                const int sub = lane & (L - 1);
                for (int step = 0; step < 32; step += 32 / L) {
                    const int rw = d.r0 + step + (lane >> lg);
                    AT sum{};
                    if (rw < d.r1) {
                        int k0 = rs[rw], k1 = rs[rw + 1];
                        bchk_range(k0, k1, d.a, d.e);
                        if (d.kind == kTileWindow) {
                            const uint16_t *lc = reinterpret_cast<const uint16_t *>(S.cols<VT, XT>(w)) - (d.a & ~7);
                            const XT *win = S.win<VT, XT>(w);
                            for (int k = k0 + sub; k < k1; k += L) sum = fma_acc(vs[k], win[bchk(lc[k], kWinMax)], sum);
                        } else {
                            const int32_t *cs = S.cols<VT, XT>(w) - (d.a & ~3);
                            for (int k = k0 + sub; k < k1; k += L) sum = fma_acc(vs[k], x[bchk(cs[k], P.n)], sum);
                        }
                    }
                    for (int m = 1; m < L; m <<= 1) sum = xor_add(sum, m);
                    if (rw < d.r1 && sub == 0) rowfn(sys, rw, sum, acc);
                    if (d.r0 + step + 32 / L >= d.r1) break;   // warp-uniform
                }
            }
            __syncwarp();
            ++count;
            Cur nx = cur;
            nx.next();
            if (nx.valid()) {
                const TileDesc dn = load_desc(P, nx.tile());
                dc = dn;
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) issue_matrix<VT, XT>(P, S, dn, w, vals);
                __syncwarp();
                issue_window<VT, XT>(P, S, dn, w, x);
            }
            cur = nx;
        }
    }
    if (acc.seg >= 0) flush_acc(B, acc);
    acc.seg = -1;
    return ok;
}


// Row function of the inner SpMM pass: p = z + beta p, q = A_lo z + beta q
// (= A_lo p) for the four right-hand sides of row i, p.q per right-hand side.
// With one lane per row the row's z, q, p and diagonal are loaded ahead
// (prefetch), before the tile's stage is waited for.
struct SpmmRow {
    const BatchParams &B;
    const PairState *st;
    int pi = -1;                 // row whose entries were loaded ahead
    float4 pz, pq, pp;
    float pdg;
    __device__ __forceinline__ void prefetch(int i) {
        pi = i;
        pz = B.p32[i];
        pq = B.q32[i];
        pp = B.pd32[i];
        pdg = B.P.diag_lo[i];
    }
    __device__ __forceinline__ void operator()(int sys, int i, float4 s4, WarpAcc<float, 4> &a) {
        const PairState *ps = st + sys * kRhs;
        const float b0 = ps[0].beta, b1 = ps[1].beta, b2 = ps[2].beta, b3 = ps[3].beta;
        const bool ahead = pi == i;
        const float dg = ahead ? pdg : B.P.diag_lo[i];
        const float4 z = ahead ? pz : B.p32[i], q0 = ahead ? pq : B.q32[i], p0 = ahead ? pp : B.pd32[i];
        const float4 qv = make_float4(fmaf(b0, q0.x, fmaf(dg, z.x, s4.x)), fmaf(b1, q0.y, fmaf(dg, z.y, s4.y)),
                                      fmaf(b2, q0.z, fmaf(dg, z.z, s4.z)), fmaf(b3, q0.w, fmaf(dg, z.w, s4.w)));
        const float4 p = make_float4(fmaf(b0, p0.x, z.x), fmaf(b1, p0.y, z.y), fmaf(b2, p0.z, z.z),
                                     fmaf(b3, p0.w, z.w));
        B.q32[i] = qv;
        B.pd32[i] = p;
        a.a[0] = fmaf(p.x, qv.x, a.a[0]);
        a.a[1] = fmaf(p.y, qv.y, a.a[1]);
        a.a[2] = fmaf(p.z, qv.z, a.a[2]);
        a.a[3] = fmaf(p.w, qv.w, a.a[3]);
    }
};

// Row function of the inner update pass: d += alpha p, r -= alpha q, z =
// dinv r (published: the SpMM of the next iteration gathers it), r.r and r.z
// per right-hand side.  A pair that is not in the inner loop (any more) keeps
// its d and r.  prefetch(i) loads row i's vectors ahead into one of two
// slots: the pass issues the next tile's loads before it finishes the
// current one, so each lane has two rows' loads in flight.
struct UpdateRow {
    const BatchParams &B;
    const PairState *st;
    int i0 = -1, i1 = -1, nxt = 0;
    float4 p0, q0, d0, r0, p1, q1, d1, r1;
    float di0 = 1.0f, di1 = 1.0f;
    __device__ __forceinline__ void prefetch(int i) {
        const float4 p = B.pd32[i], q = B.q32[i], d = B.d32[i], r = B.r32[i];
        const float di = B.P.precond ? B.P.dinv32[i] : 1.0f;
        if (nxt == 0) {
            i0 = i;
            p0 = p;
            q0 = q;
            d0 = d;
            r0 = r;
            di0 = di;
        } else {
            i1 = i;
            p1 = p;
            q1 = q;
            d1 = d;
            r1 = r;
            di1 = di;
        }
        nxt ^= 1;
    }
    __device__ __forceinline__ void operator()(int sys, int i, float4, WarpAcc<float, 8> &a) {
        const PairState *pp = st + sys * kRhs;
        const bool u0 = (pp[0].flags & kInnerActive) != 0, u1 = (pp[1].flags & kInnerActive) != 0,
                   u2 = (pp[2].flags & kInnerActive) != 0, u3 = (pp[3].flags & kInnerActive) != 0;
        const float al0 = pp[0].alpha, al1 = pp[1].alpha, al2 = pp[2].alpha, al3 = pp[3].alpha;
        float4 p, qv, d, rv;
        float di;
        if (i == i0) {
            p = p0, qv = q0, d = d0, rv = r0, di = di0;
        } else if (i == i1) {
            p = p1, qv = q1, d = d1, rv = r1, di = di1;
        } else {
            p = B.pd32[i], qv = B.q32[i], d = B.d32[i], rv = B.r32[i];
            di = B.P.precond ? B.P.dinv32[i] : 1.0f;
        }
        d = make_float4(u0 ? fmaf(al0, p.x, d.x) : d.x, u1 ? fmaf(al1, p.y, d.y) : d.y,
                        u2 ? fmaf(al2, p.z, d.z) : d.z, u3 ? fmaf(al3, p.w, d.w) : d.w);
        rv = make_float4(u0 ? fmaf(-al0, qv.x, rv.x) : rv.x, u1 ? fmaf(-al1, qv.y, rv.y) : rv.y,
                         u2 ? fmaf(-al2, qv.z, rv.z) : rv.z, u3 ? fmaf(-al3, qv.w, rv.w) : rv.w);
        B.d32[i] = d;
        B.r32[i] = rv;
        const float4 z = B.P.precond ? make_float4(di * rv.x, di * rv.y, di * rv.z, di * rv.w) : rv;
        B.p32[i] = z;
        a.a[0] = fmaf(rv.x, rv.x, a.a[0]);
        a.a[1] = fmaf(rv.y, rv.y, a.a[1]);
        a.a[2] = fmaf(rv.z, rv.z, a.a[2]);
        a.a[3] = fmaf(rv.w, rv.w, a.a[3]);
        a.a[4] = fmaf(rv.x, z.x, a.a[4]);
        a.a[5] = fmaf(rv.y, z.y, a.a[5]);
        a.a[6] = fmaf(rv.z, z.z, a.a[6]);
        a.a[7] = fmaf(rv.w, z.w, a.a[7]);
    }
};

// ---------------------------------------------------------------- kernel
template <class VT>
__global__ void __launch_bounds__(kThreads, 1) cg_batch_kernel(BatchParams B) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const Smem S = carve_smem(smem_raw);
    init_pipeline(S);
    // the block-sum area is free in this kernel: it holds the layout arrays
    int *const bsm = reinterpret_cast<int *>(S.red);
    Balance &bl = *reinterpret_cast<Balance *>(bsm + kBalHdr);
    const Params &P = B.P;
    unsigned int epoch = 0;
    uint32_t count = 0;
    int set = 0;
    PairState *st = B.state + (size_t)blockIdx.x * B.nsys * kRhs;
    const int npairs = B.nsys * kRhs;
    const VT *vlo;
    if constexpr (sizeof(VT) == 4) vlo = reinterpret_cast<const VT *>(P.vals32);
    else vlo = reinterpret_cast<const VT *>(P.vals16);
    const int nrhs = B.nrhs;

    for (int q = threadIdx.x; q < npairs; q += kThreads) {
        PairState ps{};
        const int r = q % kRhs;
        ps.flags = r < nrhs ? kOuterActive : 0;
        ps.status = r < nrhs ? CG_ENOCONV : CG_OK;
        st[q] = ps;
    }
    __syncthreads();
    auto any_flag = [&](int sys, int mask) {
        bool a = false;
        for (int r = 0; r < nrhs; ++r) a |= (st[sys * kRhs + r].flags & mask) != 0;
        return a;
    };

    for (int o = 0;; ++o) {
        // ------------------------------------------ outer residual (FP64)
        zero_wpart(B, B.cta_nsys[blockIdx.x]);
        for (int r = 0; r < nrhs; ++r) {
            WarpAcc<double, 12> acc;
            acc.seg = -1;
            auto active = [&](int sys) { return (st[sys * kRhs + r].flags & kOuterActive) != 0; };
            auto rowfn = [&](int sys, int i, double ax, WarpAcc<double, 12> &a) {
                const double bi = B.B[(size_t)r * P.n + i];
                const double ri = bi - ax;
                a.a[r] = fma(ri, ri, a.a[r]);
                a.a[4 + r] = fma(bi, bi, a.a[4 + r]);
                const float rf = (float)ri;
                const float zf = P.precond ? P.dinv32[i] * rf : rf;
                float4 v = B.r32[i];
                f4set(v, r, rf);
                B.r32[i] = v;
                v = B.p32[i];
                f4set(v, r, zf);
                B.p32[i] = v;
                v = B.pd32[i];
                f4set(v, r, zf);
                B.pd32[i] = v;
                v = B.q32[i];
                f4set(v, r, 0.0f);
                B.q32[i] = v;
                v = B.d32[i];
                f4set(v, r, 0.0f);
                B.d32[i] = v;
                a.a[8 + r] = fma((double)rf, (double)zf, a.a[8 + r]);
            };
            if (!batch_pass<double, double, double>(B, S, count, P.vals, B.xw + (size_t)r * B.xstride,
                                                    static_tiles(B, active), rowfn, acc))
                goto out;
        }
        combine_segments(B, set, 12);
        if (!grid_barrier(P, epoch, S)) goto out;
        {
            int inner_any = 0;
            for (int q = threadIdx.x; q < npairs; q += kThreads) {
                PairState ps = st[q];
                const int sys = q / kRhs, r = q % kRhs;
                ps.flags &= ~kRanInner;
                if (ps.flags & kOuterActive) {
                    const double rr = system_total<double>(B, set, sys, r);
                    const double bb = system_total<double>(B, set, sys, 4 + r);
                    const double rz = system_total<double>(B, set, sys, 8 + r);
                    if (o == 0) ps.bnorm = sqrt(bb);
                    ps.relres = ps.bnorm > 0.0 ? sqrt(rr) / ps.bnorm : 0.0;
                    if (!finite_bits(rr) || !finite_bits(bb) || !finite_bits(rz)) {
                        ps.status = CG_ENAN;
                        ps.flags = 0;
                    } else if (ps.bnorm == 0.0) {  // b = 0: x = 0 in the update below
                        ps.status = CG_OK;
                        ps.flags = kRanInner;
                        ps.relres = 0.0;
                        ps.rho = -1.0;
                    } else if (rr <= (B.tol * ps.bnorm) * (B.tol * ps.bnorm)) {
                        ps.status = CG_OK;
                        ps.flags = 0;
                    } else if (o == B.max_outer || ps.iters >= B.maxit) {
                        ps.status = CG_ENOCONV;
                        ps.flags = 0;
                    } else if (!(rz > 0.0)) {
                        ps.status = CG_EBREAKDOWN;
                        ps.flags = 0;
                    } else {
                        ps.flags = kOuterActive | kInnerActive | kRanInner;
                        ps.rho = rz;
                        ps.beta = 0.0f;   // p_1 = z_0, q_1 = A z_0
                        ps.target2 = B.inner_tol * B.inner_tol * rr;
                        ps.outer = o + 1;
                        inner_any = 1;
                    }
                }
                st[q] = ps;
            }
            set ^= 1;
            if (__syncthreads_or(inner_any)) {
                // ------------------------------------------ inner CG (FP32, 4 rhs)
                auto active = [&](int sys) { return any_flag(sys, kInnerActive); };
                if (B.balance) compute_balance(B, active, bsm);
                else if (threadIdx.x == 0) bl.dyn = 0;
                __syncthreads();
                for (int k = 1;; ++k) {
                    const bool dyn = bl.dyn != 0;
                    const int nloc = dyn ? bl.nloc : B.cta_nsys[blockIdx.x];
                    // p = z + beta p, q = A_lo z + beta q (= A_lo p); p.q
                    // (the SpMM gathers z: A p = A z + beta A p_old)
                    zero_wpart(B, nloc);
                    {
                        WarpAcc<float, 4> acc;
                        acc.seg = -1;
                        SpmmRow rowfn{B, st};
                        const bool ok =
                            dyn ? batch_pass<VT, float4, float4>(B, S, count, vlo, B.p32, balanced_tiles(B, bl), rowfn, acc)
                                : batch_pass<VT, float4, float4>(B, S, count, vlo, B.p32, static_tiles(B, active), rowfn,
                                                                 acc);
                        if (!ok) goto out;
                    }
                    if (dyn) combine_segments_dyn(B, set, 4, nloc);
                    else combine_segments(B, set, 4);
                    if (!grid_barrier(P, epoch, S)) goto out;
                    int left_now = 0;
                    for (int q = threadIdx.x; q < npairs; q += kThreads) {
                        PairState ps = st[q];
                        ps.alpha = 0.0f;
                        if (ps.flags & kInnerActive) {
                            float sg;
                            if (dyn) {
                                const int sl[1] = {q % kRhs};
                                float o[1];
                                system_totals_dyn<1>(B, set, bl.total, q / kRhs, sl, o);
                                sg = o[0];
                            } else {
                                sg = system_total<float>(B, set, q / kRhs, q % kRhs);
                            }
                            if (!(sg > 0.0f) || !isfinite(sg)) {
                                ps.flags &= ~kInnerActive;  // keep d so far
                                left_now = 1;
                            } else {
                                ps.alpha = (float)ps.rho / sg;
                            }
                        }
                        st[q] = ps;
                    }
                    __syncthreads();
                    set ^= 1;
                    // d += alpha p, r -= alpha q, z = dinv r (gathered by the next SpMM:
                    // every gather of this one is over); r.r, r.z
                    zero_wpart(B, nloc);
                    {
                        WarpAcc<float, 8> acc;
                        acc.seg = -1;
                        UpdateRow rowfn{B, st};
                        const bool ok =
                            dyn ? batch_pass<VT, float4, float4>(B, S, count, (const VT *)nullptr,
                                                                 (const float4 *)nullptr, balanced_tiles(B, bl), rowfn,
                                                                 acc)
                                : batch_pass<VT, float4, float4>(B, S, count, (const VT *)nullptr,
                                                                 (const float4 *)nullptr, static_tiles(B, active), rowfn,
                                                                 acc);
                        if (!ok) goto out;
                    }
                    if (dyn) combine_segments_dyn(B, set, 8, nloc);
                    else combine_segments(B, set, 8);
                    if (!grid_barrier(P, epoch, S)) goto out;
                    int left = 0;
                    for (int q = threadIdx.x; q < npairs; q += kThreads) {
                        PairState ps = st[q];
                        ps.beta = 0.0f;
                        if (ps.flags & kInnerActive) {
                            const int r = q % kRhs;
                            float rr, rz;
                            if (dyn) {
                                const int sl[2] = {r, 4 + r};
                                float o[2];
                                system_totals_dyn<2>(B, set, bl.total, q / kRhs, sl, o);
                                rr = o[0];
                                rz = o[1];
                            } else {
                                rr = system_total<float>(B, set, q / kRhs, r);
                                rz = system_total<float>(B, set, q / kRhs, 4 + r);
                            }
                            ++ps.iters;
                            if (!isfinite(rr) || !isfinite(rz) || !(rz > 0.0f) || (double)rr <= ps.target2 ||
                                k >= B.max_inner || ps.iters >= B.maxit) {
                                ps.flags &= ~kInnerActive;
                                left_now = 1;
                            } else {
                                ps.beta = rz / (float)ps.rho;
                                ps.rho = rz;
                                left = 1;
                            }
                        }
                        st[q] = ps;
                    }
                    set ^= 1;
                    if (!__syncthreads_or(left)) break;
                    // a pair left the inner loop: its system may have, so re-split
                    if (B.balance && __syncthreads_or(left_now)) compute_balance(B, active, bsm);
                }
            }
        }

        // ------------------------------------------ x += d (FP64)
        {
            int ran = 0, outer_left = 0;
            for (int q = threadIdx.x; q < npairs; q += kThreads) {
                ran |= (st[q].flags & kRanInner) != 0;
                outer_left |= (st[q].flags & kOuterActive) != 0;
            }
            if (__syncthreads_or(ran)) {
                WarpAcc<float, 0> acc;
                acc.seg = -1;
                auto active = [&](int sys) { return any_flag(sys, kRanInner); };
                auto rowfn = [&](int sys, int i, float4, WarpAcc<float, 0> &) {
                    const float4 d = B.d32[i];
                    for (int r = 0; r < nrhs; ++r) {
                        const PairState &ps = st[sys * kRhs + r];
                        if (!(ps.flags & kRanInner)) continue;
                        double &x = B.xw[(size_t)r * B.xstride + i];
                        x = ps.rho < 0.0 ? 0.0 : x + (double)f4c(d, r);
                    }
                };
                if (!batch_pass<VT, float4, float4>(B, S, count, (const VT *)nullptr, (const float4 *)nullptr,
                                                    static_tiles(B, active),
                                                    rowfn, acc))
                    goto out;
            }
            const bool more = __syncthreads_or(outer_left) != 0;
            if (!grid_barrier(P, epoch, S)) goto out;
            if (!more) break;
        }
    }

    if (blockIdx.x == 0) {
        for (int q = threadIdx.x; q < npairs; q += kThreads) {
            const PairState &ps = st[q];
            cg_batch_result res{};
            res.iters = ps.iters;
            res.outer = ps.outer;
            res.status = ps.status;
            res.relres = ps.relres;
            B.results[q] = res;
        }
    }
out:
    // no copy is left in flight: every pass waits for each tile it issued
    __syncthreads();
}

}  // namespace

// =================================================================== host

struct cg_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    cg_opts opts{};
    int32_t nsys = 0, n = 0, ctas = 0, nseg = 0, xstride = 0, ntiles = 0;
    int64_t nnz = 0;
    double inner_tol = 1e-3;
    int use_gather = 0;                 // tuned: 1 = gather tiles instead of x-windows
    int lanes_per_row = 1;              // tuned: SpMM lanes per row (rows per warp step 32 / this)
    int static_split = 0;               // 1: the inner loop keeps the creation-time split
    std::vector<int32_t> sys_rows;
    // device
    int32_t *rowptr = nullptr, *colidx = nullptr, *tile_sys = nullptr, *cta_tile = nullptr;
    int32_t *cta_sys0 = nullptr, *cta_nsys = nullptr, *cta_seg0 = nullptr, *sys_seg0 = nullptr;
    int32_t *sys_tile0 = nullptr, *bal = nullptr;
    int4 *sinf = nullptr;
    double *segdyn = nullptr;
    int4 *tiles_win = nullptr, *tiles_gather = nullptr, *segs = nullptr;
    uint16_t *lcol = nullptr, *vals16 = nullptr;
    double *vals = nullptr, *xw = nullptr, *wpart = nullptr, *segpart = nullptr;
    float *vals32 = nullptr, *diag_lo = nullptr, *dinv32 = nullptr;
    float4 *r32 = nullptr, *z32 = nullptr, *p32 = nullptr, *q32 = nullptr, *d32 = nullptr;
    float4 *pd32 = nullptr;
    PairState *state = nullptr;
    cg_batch_result *results = nullptr;
    unsigned int *bar = nullptr;
    DevStatus *st = nullptr;
    cg_batch_result *results_host = nullptr;  // pinned
    DevStatus *st_host = nullptr;             // pinned
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<void *> allocs;
    int last_nrhs = 0;
};

namespace {

template <class T>
int bdev_alloc(cg_batch *h, T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    void *v = nullptr;
    cudaError_t e = cudaMalloc(&v, count * sizeof(T));
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? CG_ENOMEM : CG_ECUDA;
    h->allocs.push_back(v);
    *p = static_cast<T *>(v);
    return CG_OK;
}

template <class T>
int bupload(T *dst, const std::vector<T> &src) {
    if (src.empty()) return CG_OK;
    return cudaMemcpy(dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice) == cudaSuccess ? CG_OK
                                                                                                       : CG_ECUDA;
}

void batch_free(cg_batch *h) {
    if (!h) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    for (void *p : h->allocs) cudaFree(p);
    if (h->results_host) cudaFreeHost(h->results_host);
    if (h->st_host) cudaFreeHost(h->st_host);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    cudaSetDevice(prev);
    delete h;
}

BatchParams batch_params(const cg_batch *h, const double *Bm, int nrhs, double tol, int maxit) {
    BatchParams B{};
    Params &P = B.P;
    P.n = h->n;
    P.rowptr = h->rowptr;
    P.colidx = h->colidx;
    P.vals = h->vals;
    P.tiles = h->use_gather ? h->tiles_gather : h->tiles_win;
    P.lcol = h->lcol;
    P.segs = h->segs;
    P.cta_tile = h->cta_tile;
    P.vals32 = h->vals32;
    P.vals16 = reinterpret_cast<const __nv_bfloat16 *>(h->vals16);
    P.diag_lo = h->diag_lo;
    P.dinv32 = h->dinv32;
    P.bar = h->bar;
    P.st = h->st;
    P.wait_ns = (unsigned long long)(h->opts.wait_limit_s * 1e9);
    P.phantom = h->opts.debug_phantom_arrivals;
    P.precond = h->opts.precond;
    P.evict_first = 1;
    B.tile_sys = h->tile_sys;
    B.cta_sys0 = h->cta_sys0;
    B.cta_nsys = h->cta_nsys;
    B.cta_seg0 = h->cta_seg0;
    B.sys_seg0 = h->sys_seg0;
    B.nsys = h->nsys;
    B.nrhs = nrhs;
    B.nseg = h->nseg;
    B.lanes_per_row = h->lanes_per_row;
    B.tol = tol;
    B.inner_tol = h->inner_tol;
    B.maxit = maxit;
    B.max_outer = h->opts.max_outer;
    B.max_inner = h->opts.max_inner > 0 ? h->opts.max_inner : std::max(h->n, 1);
    B.B = Bm;
    B.xw = h->xw;
    B.xstride = h->xstride;
    B.r32 = h->r32;
    B.z32 = h->z32;
    B.p32 = h->p32;
    B.pd32 = h->pd32;
    B.q32 = h->q32;
    B.d32 = h->d32;
    B.wpart = h->wpart;
    B.segpart = h->segpart;
    B.state = h->state;
    B.results = h->results;
    B.sys_tile0 = h->sys_tile0;
    B.bal = h->bal;
    B.sinf = h->sinf;
    B.segdyn = h->segdyn;
    B.balance = (h->ctas <= kMaxBalCtas && !h->static_split) ? 1 : 0;
    return B;
}

constexpr int kBatchSmem = kSmemBytes;

int batch_enqueue(cg_batch *h, const double *Bm, double *X, int nrhs, double tol, int maxit, bool copy_back) {
    const size_t col = sizeof(double) * (size_t)h->n, pitch = sizeof(double) * (size_t)h->xstride;
    cudaError_t e = cudaMemcpy2DAsync(h->xw, pitch, X, col, col, (size_t)nrhs, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->bar, 0, sizeof(unsigned int), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->st, 0, sizeof(DevStatus), h->stream);
    if (e == cudaSuccess) {
        BatchParams B = batch_params(h, Bm, nrhs, tol, maxit);
        void *args[] = {&B};
        const void *kern = h->opts.inner_values == CG_VALUES_BF16 ? (const void *)cg_batch_kernel<__nv_bfloat16>
                                                                  : (const void *)cg_batch_kernel<float>;
        e = cudaLaunchCooperativeKernel(kern, dim3(h->ctas), dim3(kThreads), args, (size_t)kBatchSmem, h->stream);
    }
    if (e == cudaSuccess && copy_back)
        e = cudaMemcpy2DAsync(X, col, h->xw, pitch, col, (size_t)nrhs, cudaMemcpyDeviceToDevice, h->stream);
    h->last_nrhs = nrhs;
    return e == cudaSuccess ? CG_OK : CG_ECUDA;
}

int batch_collect(cg_batch *h, cg_batch_result *results) {
    const size_t nres = (size_t)h->nsys * kRhs;
    cudaError_t e = cudaMemcpyAsync(h->results_host, h->results, sizeof(cg_batch_result) * nres,
                                    cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->st_host, h->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return CG_ECUDA;
    if (h->st_host->status != 0) return h->st_host->status;  // a bounded wait ran out
    int worst = CG_OK;
    for (int s = 0; s < h->nsys; ++s) {
        for (int r = 0; r < h->last_nrhs; ++r) {
            const cg_batch_result &res = h->results_host[(size_t)s * kRhs + r];
            if (results) results[(size_t)s * h->last_nrhs + r] = res;
            if (res.status != CG_OK && worst == CG_OK) worst = res.status;
        }
    }
    return worst;
}

}  // namespace

long long gbcg::bounds_faults_batch() { return read_bounds_faults(); }

extern "C" {

int cg_batch_create(const cg_csr *systems, int32_t nsys, const cg_opts *opts_in, void *stream, cg_batch **out) {
    NvtxRange nvtx("gbcg.batch_create");
    if (!out) return CG_EINVAL;
    *out = nullptr;
    if (!systems || nsys < 1) return CG_EINVAL;
    cg_opts opts;
    if (opts_in) opts = *opts_in;
    else cg_opts_default(&opts);
    if (opts.inner_values == CG_VALUES_FP64) opts.inner_values = CG_VALUES_FP32;
    if (opts.inner_values != CG_VALUES_FP32 && opts.inner_values != CG_VALUES_BF16) return CG_EINVAL;
    if (opts.precond != CG_PRECOND_NONE && opts.precond != CG_PRECOND_JACOBI) return CG_EINVAL;
    if (!(opts.wait_limit_s > 0.0) || !std::isfinite(opts.wait_limit_s) || opts.wait_limit_s > 3600.0) return CG_EINVAL;
    if (opts.inner_tol == 0.0) opts.inner_tol = opts.inner_values == CG_VALUES_BF16 ? 1e-2 : 1e-3;
    if (!(opts.inner_tol > 0.0 && opts.inner_tol < 1.0) || opts.max_outer < 1 || opts.max_inner < 0 ||
        opts.debug_phantom_arrivals < 0 || opts.debug_phantom_arrivals > 1024)
        return CG_EINVAL;

    // ---- concatenate the systems into one block-diagonal CSR (validated)
    std::vector<int32_t> rowptr(1, 0), colidx, sys_rows(1, 0);
    std::vector<double> vals;
    int64_t total_n = 0, total_nnz = 0;
    for (int s = 0; s < nsys; ++s) {
        const cg_csr &A = systems[s];
        if (A.n < 0 || A.nnz < 0 || (A.mem != CG_MEM_HOST && A.mem != CG_MEM_DEVICE) || !A.rowptr ||
            (A.nnz > 0 && (!A.colidx || !A.vals)))
            return CG_EINVAL;
        total_n += A.n;
        total_nnz += A.nnz;
        if (total_n > (int64_t)INT32_MAX - 64 || total_nnz > (int64_t)INT32_MAX - 64) return CG_EINVAL;
    }
    rowptr.reserve((size_t)total_n + 1);
    colidx.reserve((size_t)total_nnz);
    vals.reserve((size_t)total_nnz);
    for (int s = 0; s < nsys; ++s) {
        const cg_csr &A = systems[s];
        std::vector<int32_t> rp(A.n + 1), ci(A.nnz);
        std::vector<double> va(A.nnz);
        if (A.mem == CG_MEM_DEVICE) {
            if (cudaMemcpy(rp.data(), A.rowptr, sizeof(int32_t) * (A.n + 1), cudaMemcpyDeviceToHost) != cudaSuccess)
                return CG_EINVAL;
            if (A.nnz > 0 &&
                (cudaMemcpy(ci.data(), A.colidx, sizeof(int32_t) * A.nnz, cudaMemcpyDeviceToHost) != cudaSuccess ||
                 cudaMemcpy(va.data(), A.vals, sizeof(double) * A.nnz, cudaMemcpyDeviceToHost) != cudaSuccess))
                return CG_EINVAL;
        } else {
            std::memcpy(rp.data(), A.rowptr, sizeof(int32_t) * (A.n + 1));
            if (A.nnz > 0) {
                std::memcpy(ci.data(), A.colidx, sizeof(int32_t) * A.nnz);
                std::memcpy(va.data(), A.vals, sizeof(double) * A.nnz);
            }
        }
        if (rp[0] != 0 || (int64_t)rp[A.n] != A.nnz) return CG_EINVAL;
        for (int32_t i = 0; i < A.n; ++i)
            if (rp[i + 1] < rp[i]) return CG_EINVAL;
        const int32_t roff = sys_rows.back(), koff = rowptr.back();
        for (int64_t k = 0; k < A.nnz; ++k) {
            if (ci[k] < 0 || ci[k] >= A.n) return CG_EINVAL;
            colidx.push_back(ci[k] + roff);
            vals.push_back(va[k]);
        }
        for (int32_t i = 1; i <= A.n; ++i) rowptr.push_back(rp[i] + koff);
        sys_rows.push_back(roff + A.n);
    }
    const int32_t n = sys_rows.back();
    const int64_t nnz = (int64_t)colidx.size();
    InnerMatrix inner = build_inner(n, rowptr, colidx, vals, opts.inner_values == CG_VALUES_FP32 ? 1 : 2);
    if (opts.precond == CG_PRECOND_JACOBI)
        for (int32_t i = 0; i < n; ++i)
            if (!(inner.diag[i] > 0.0f) || !std::isfinite(inner.diag[i])) return CG_EINVAL;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CG_ECUDA;
    cg_batch *h = new (std::nothrow) cg_batch();
    if (!h) return CG_ENOMEM;
    h->device = dev;
    h->stream = static_cast<cudaStream_t>(stream);
    h->opts = opts;
    h->nsys = nsys;
    h->n = n;
    h->nnz = nnz;
    h->inner_tol = opts.inner_tol;
    h->sys_rows = sys_rows;
    auto fail = [&](int code) {
        batch_free(h);
        return code;
    };

    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return fail(CG_ECUDA);
    if (cudaFuncSetAttribute((const void *)cg_batch_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kBatchSmem) != cudaSuccess ||
        cudaFuncSetAttribute((const void *)cg_batch_kernel<__nv_bfloat16>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, kBatchSmem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cg_batch_kernel<float>, kThreads, kBatchSmem) !=
            cudaSuccess ||
        per_sm < 1)
        return fail(CG_ECUDA);
    int ctas = opts.grid_ctas > 0 ? std::min(opts.grid_ctas, sms * per_sm) : sms;
    int max_tile = 0;
    BatchPlan bp = plan_batch(rowptr, sys_rows, ctas, &max_tile);
    if (bp.max_nsys_per_cta > kMaxSegPerCta) return fail(CG_EINVAL);  // too many tiny systems per CTA
    TilePlan tp = plan_windows(n, rowptr, colidx, bp.tiles);
    std::vector<I4> desc_gather = tp.desc;
    for (size_t t = 0; t + 1 < bp.tiles.size(); ++t) {
        I4 &d1 = desc_gather[2 * t + 1];
        if (d1.w == kTileWindow) d1 = mk4(0, 0, 0, kTileGather);
    }
    // first tile of each system (tiles are in system order)
    std::vector<int32_t> sys_tile0((size_t)nsys + 1, 0);
    for (int32_t s : bp.tile_sys) ++sys_tile0[(size_t)s + 1];
    for (int s = 0; s < nsys; ++s) sys_tile0[(size_t)s + 1] += sys_tile0[s];
    h->ctas = ctas;
    h->nseg = (int)bp.seg_cta.size();
    h->ntiles = (int)bp.tile_sys.size();
    h->xstride = ((n + 3) / 4) * 4 + 4;

    const size_t pad = 32;
    int rc = CG_OK;
    if ((rc = bdev_alloc(h, &h->rowptr, (size_t)n + 1 + pad)) || (rc = bdev_alloc(h, &h->colidx, (size_t)nnz + pad)) ||
        (rc = bdev_alloc(h, &h->vals, (size_t)nnz + pad)) || (rc = bdev_alloc(h, &h->lcol, (size_t)nnz + pad)) ||
        (rc = bdev_alloc(h, &h->tiles_win, tp.desc.size())) ||
        (rc = bdev_alloc(h, &h->tiles_gather, desc_gather.size())) ||
        (rc = bdev_alloc(h, &h->segs, tp.segs.size())) || (rc = bdev_alloc(h, &h->tile_sys, bp.tile_sys.size())) ||
        (rc = bdev_alloc(h, &h->cta_tile, bp.cut.size())) || (rc = bdev_alloc(h, &h->cta_sys0, bp.cta_sys0.size())) ||
        (rc = bdev_alloc(h, &h->cta_nsys, bp.cta_nsys.size())) ||
        (rc = bdev_alloc(h, &h->cta_seg0, bp.cta_seg0.size())) ||
        (rc = bdev_alloc(h, &h->sys_seg0, bp.sys_seg0.size())) || (rc = bdev_alloc(h, &h->diag_lo, (size_t)n + 1)) ||
        (rc = bdev_alloc(h, &h->sys_tile0, sys_tile0.size())) ||
        (rc = bdev_alloc(h, &h->bal, (size_t)ctas * 2 * ((size_t)nsys + 1))) ||
        (rc = bdev_alloc(h, &h->sinf, (size_t)ctas * nsys)) ||
        (rc = bdev_alloc(h, &h->segdyn, (size_t)2 * ctas * kMaxSegPerCta * kSlots)) ||
        (rc = bdev_alloc(h, &h->xw, (size_t)kRhs * h->xstride)) ||
        (rc = bdev_alloc(h, &h->r32, (size_t)n + 1)) || (rc = bdev_alloc(h, &h->p32, (size_t)n + pad)) ||
        (rc = bdev_alloc(h, &h->pd32, (size_t)n + 1)) ||
        (rc = bdev_alloc(h, &h->q32, (size_t)n + 1)) || (rc = bdev_alloc(h, &h->d32, (size_t)n + 1)) ||
        (rc = bdev_alloc(h, &h->wpart, (size_t)ctas * kWarps * kMaxSegPerCta * kSlots)) ||
        (rc = bdev_alloc(h, &h->segpart, (size_t)2 * std::max(h->nseg, 1) * kSlots)) ||
        (rc = bdev_alloc(h, &h->state, (size_t)ctas * nsys * kRhs)) ||
        (rc = bdev_alloc(h, &h->results, (size_t)nsys * kRhs)) || (rc = bdev_alloc(h, &h->bar, 64)) ||
        (rc = bdev_alloc(h, &h->st, 1)))
        return fail(rc);
    if (opts.precond == CG_PRECOND_JACOBI) {
        if ((rc = bdev_alloc(h, &h->z32, (size_t)n + 1)) || (rc = bdev_alloc(h, &h->dinv32, (size_t)n + 1)))
            return fail(rc);
    } else {
        h->z32 = h->r32;
    }
    if (opts.inner_values == CG_VALUES_FP32) {
        if ((rc = bdev_alloc(h, &h->vals32, (size_t)nnz + pad))) return fail(rc);
    } else {
        if ((rc = bdev_alloc(h, &h->vals16, (size_t)nnz + pad))) return fail(rc);
    }
    if (cudaMallocHost(&h->results_host, sizeof(cg_batch_result) * (size_t)nsys * kRhs) != cudaSuccess ||
        cudaMallocHost(&h->st_host, sizeof(DevStatus)) != cudaSuccess)
        return fail(CG_ENOMEM);
    if (cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess) return fail(CG_ECUDA);

    cudaError_t e = cudaMemset(h->rowptr, 0, sizeof(int32_t) * (n + 1 + pad));
    if (e == cudaSuccess) e = cudaMemset(h->colidx, 0, sizeof(int32_t) * (nnz + pad));
    if (e == cudaSuccess) e = cudaMemset(h->vals, 0, sizeof(double) * (nnz + pad));
    if (e == cudaSuccess) e = cudaMemset(h->p32, 0, sizeof(float4) * (n + pad));
    if (e == cudaSuccess) e = cudaMemset(h->xw, 0, sizeof(double) * kRhs * h->xstride);
    if (e != cudaSuccess) return fail(CG_ECUDA);
    std::vector<uint16_t> lcol(tp.lcol.begin(), tp.lcol.begin() + std::min(tp.lcol.size(), (size_t)nnz + pad));
    if ((rc = bupload(h->rowptr, rowptr)) || (rc = bupload(h->colidx, colidx)) || (rc = bupload(h->vals, vals)) ||
        (rc = bupload(h->lcol, lcol)) || (rc = bupload(reinterpret_cast<I4 *>(h->tiles_win), tp.desc)) ||
        (rc = bupload(reinterpret_cast<I4 *>(h->tiles_gather), desc_gather)) ||
        (rc = bupload(reinterpret_cast<I4 *>(h->segs), tp.segs)) ||
        (rc = bupload(h->tile_sys, bp.tile_sys)) || (rc = bupload(h->cta_tile, bp.cut)) ||
        (rc = bupload(h->cta_sys0, bp.cta_sys0)) || (rc = bupload(h->cta_nsys, bp.cta_nsys)) ||
        (rc = bupload(h->cta_seg0, bp.cta_seg0)) || (rc = bupload(h->sys_seg0, bp.sys_seg0)) ||
        (rc = bupload(h->sys_tile0, sys_tile0)) ||
        (rc = bupload(h->diag_lo, inner.diag)))
        return fail(rc);
    if (opts.inner_values == CG_VALUES_FP32) {
        std::vector<float> v32 = inner.vals32;
        v32.resize((size_t)nnz + pad, 0.0f);
        if ((rc = bupload(h->vals32, v32))) return fail(rc);
    } else {
        std::vector<uint16_t> v16 = inner.vals16;
        v16.resize((size_t)nnz + pad, 0);
        if ((rc = bupload(h->vals16, v16))) return fail(rc);
    }
    if (opts.precond == CG_PRECOND_JACOBI) {
        std::vector<float> di(n);
        for (int32_t i = 0; i < n; ++i) di[i] = 1.0f / inner.diag[i];
        if ((rc = bupload(h->dinv32, di))) return fail(rc);
    }
    *out = h;
    return CG_OK;
}

int cg_batch_enqueue(cg_batch *h, const double *B, double *X, int32_t nrhs, double tol, int32_t maxit) {
    NvtxRange nvtx("gbcg.batch_enqueue");
    if (!h || !B || !X || nrhs < 1 || nrhs > kRhs || !(tol >= 0.0) || !std::isfinite(tol)) return CG_EINVAL;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != h->device) cudaSetDevice(h->device);
    const int rc = batch_enqueue(h, B, X, nrhs, tol, maxit > 0 ? maxit : std::max(h->n, 1), true);
    if (prev >= 0 && prev != h->device) cudaSetDevice(prev);
    return rc;
}

int cg_batch_results(cg_batch *h, cg_batch_result *results) {
    if (!h) return CG_EINVAL;
    return batch_collect(h, results);
}

int cg_batch_solve(cg_batch *h, const double *B, double *X, int32_t nrhs, double tol, int32_t maxit,
                   cg_batch_result *results, double *kernel_ms) {
    NvtxRange nvtx("gbcg.batch_solve");
    if (!h || !B || !X || nrhs < 1 || nrhs > kRhs || !(tol >= 0.0) || !std::isfinite(tol)) return CG_EINVAL;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != h->device) cudaSetDevice(h->device);
    int rc = CG_OK;
    if (cudaEventRecord(h->ev0, h->stream) != cudaSuccess) rc = CG_ECUDA;
    if (rc == CG_OK) rc = batch_enqueue(h, B, X, nrhs, tol, maxit > 0 ? maxit : std::max(h->n, 1), true);
    if (rc == CG_OK && cudaEventRecord(h->ev1, h->stream) != cudaSuccess) rc = CG_ECUDA;
    if (rc == CG_OK) rc = batch_collect(h, results);
    if (kernel_ms) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, h->ev0, h->ev1);
        *kernel_ms = ms;
    }
    if (prev >= 0 && prev != h->device) cudaSetDevice(prev);
    return rc;
}

int cg_batch_tune(cg_batch *h, const double *B, double *X, int32_t nrhs, double tol, cg_batch_tuning *choice) {
    NvtxRange nvtx("gbcg.batch_tune");
    if (!h || !B || !X || nrhs < 1 || nrhs > kRhs) return CG_EINVAL;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != h->device) cudaSetDevice(h->device);
    const double tols[] = {1e-2, 3e-3, 1e-3, 1e-4};
    const int lanes[] = {1, 2, 4};
    double best_ms = 1e300, best_tol = h->inner_tol;
    int best_gather = h->use_gather, best_lanes = h->lanes_per_row, tried = 0, rc = CG_OK;
    for (int gather = 0; gather < 2 && rc == CG_OK; ++gather) {
        for (int L : lanes) {
            for (double it : tols) {
                if (h->opts.inner_values == CG_VALUES_BF16 && it < 1e-3) continue;  // beyond BF16's refinement
                h->inner_tol = it;
                h->use_gather = gather;
                h->lanes_per_row = L;
                float ms = 0.0f;
                // x0 from X, result not copied back: the caller's X is left as it was
                if (cudaEventRecord(h->ev0, h->stream) != cudaSuccess) { rc = CG_ECUDA; break; }
                int r = batch_enqueue(h, B, X, nrhs, tol, std::max(h->n, 1), false);
                if (r == CG_OK && cudaEventRecord(h->ev1, h->stream) != cudaSuccess) r = CG_ECUDA;
                if (r == CG_OK) r = batch_collect(h, nullptr);
                if (r == CG_ECUDA || r == CG_ETIMEOUT) { rc = r; break; }
                cudaEventElapsedTime(&ms, h->ev0, h->ev1);
                ++tried;
                if (r == CG_OK && ms < best_ms) {
                    best_ms = ms;
                    best_tol = it;
                    best_gather = gather;
                    best_lanes = L;
                }
            }
            if (rc != CG_OK) break;
        }
    }
    h->inner_tol = best_tol;
    h->use_gather = best_gather;
    h->lanes_per_row = best_lanes;
    if (choice) {
        choice->inner_tol = best_tol;
        choice->gather_tiles = best_gather;
        choice->trials = tried;
        choice->best_ms = best_ms < 1e300 ? best_ms : -1.0;
        choice->lanes_per_row = best_lanes;
        choice->static_split = h->static_split;
    }
    if (prev >= 0 && prev != h->device) cudaSetDevice(prev);
    return rc;
}

int cg_batch_set_tuning(cg_batch *h, const cg_batch_tuning *choice) {
    if (!h || !choice) return CG_EINVAL;
    if (!(choice->inner_tol > 0.0 && choice->inner_tol < 1.0) || (choice->gather_tiles != 0 && choice->gather_tiles != 1) ||
        (choice->lanes_per_row != 1 && choice->lanes_per_row != 2 && choice->lanes_per_row != 4) ||
        (choice->static_split != 0 && choice->static_split != 1))
        return CG_EINVAL;
    h->inner_tol = choice->inner_tol;
    h->use_gather = choice->gather_tiles;
    h->lanes_per_row = choice->lanes_per_row;
    h->static_split = choice->static_split;
    return CG_OK;
}

void cg_batch_destroy(cg_batch *h) { batch_free(h); }

}  // extern "C"
