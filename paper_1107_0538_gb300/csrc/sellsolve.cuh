// The FP64 building blocks of the SELL-32 solve kernels (1024 threads a CTA,
// one per SM), shared by the CG solves and the flexible-CG iteration: row
// sums of a slice, and fixed-order sums over the CTA and over the grid.
#pragma once

#include "cg_device.cuh"
#include "sell.cuh"

namespace gbcg {

constexpr int kSellSolveThreads = 1024;
constexpr int kSellUnrollMem = 18;   // loads in flight per row where rows are not held in registers

// Sums over the CTA in a fixed order with the FP64 work spread over the four
// SM sub-partitions (warp w issues on sub-partition w mod 4; one warp-wide
// FP64 add occupies a sub-partition's FP64 pipe for ~64 cycles, so the number
// of adds on the busiest sub-partition is the cost).  Quarter g of 32
// partials per lane is added by warp g and folded by a butterfly; lane j of
// warp 0 then adds the four quarter sums of value j.  Thread 0 ends with the
// totals, the same bits in every CTA and every run.
//
// Two values share one butterfly: lanes 0-15 fold value 0 and lanes 16-31
// value 1 after the first exchange.
template <int NV>
__device__ __forceinline__ void fold_quarter(double (&t)[NV], double *quarter, int g) {
    const int lane = threadIdx.x & 31;
    if constexpr (NV == 2) {
        const bool lo = lane < 16;
        const double keep = lo ? t[0] : t[1];
        double u = keep + __shfl_xor_sync(0xffffffffu, lo ? t[1] : t[0], 16);
#pragma unroll
        for (int m = 8; m >= 1; m >>= 1) u += __shfl_xor_sync(0xffffffffu, u, m);
        if (lane == 0) quarter[g] = u;
        if (lane == 16) quarter[4 + g] = u;
    } else {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            const double u = warp_sum(t[j]);
            if (lane == 0) quarter[4 * j + g] = u;
        }
    }
}

// Thread 0 (and every lane of warp 0) gets the totals of the four quarters.
template <int NV>
__device__ __forceinline__ void add_quarters(double (&v)[NV], const double *quarter) {
    const int lane = threadIdx.x & 31;
    double t = 0.0;
    if (lane < NV) {
        const double *q = quarter + 4 * lane;
        t = (q[0] + q[1]) + (q[2] + q[3]);
    }
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = __shfl_sync(0xffffffffu, t, j);
}

template <int NV>
__device__ __forceinline__ void block_sum_1k(double (&v)[NV], double *red, double *quarter) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; ++j) red[j * kSellSolveThreads + threadIdx.x] = v[j];
    __syncthreads();
    if (w < 4) {
        double t[NV];
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            // 8 partials per lane, added as a tree (depth 3, not a chain of 7)
            const double *src = red + j * kSellSolveThreads + 32 * w + lane;
            static_assert(kSellSolveThreads / 128 == 8, "8 partials per lane");
            t[j] = ((src[0] + src[128]) + (src[256] + src[384])) + ((src[512] + src[640]) + (src[768] + src[896]));
        }
        fold_quarter<NV>(t, quarter, w);
    }
    __syncthreads();
    if (w == 0) add_quarters<NV>(v, quarter);
}

// Grid totals of the partials of barrier set `set`: warp g < 4 adds the
// partials of CTAs g*32 + lane + 128 u, then as above.  Every CTA computes
// the same bits.
template <int NV>
__device__ __forceinline__ void grid_totals_1k(const Params &P, int set, double (&out)[NV], double *quarter) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int G = (int)gridDim.x;
    if (w < 4) {
        const double *src = P.partials + (size_t)set * G * kRedSlots;
        double t[NV];
        const int m0 = 32 * w + lane;
#pragma unroll
        for (int j = 0; j < NV; ++j) t[j] = m0 < G ? __ldcg(src + (size_t)m0 * kRedSlots + j) : 0.0;
        for (int m = m0 + 128; m - lane < G; m += 128) {
#pragma unroll
            for (int j = 0; j < NV; ++j) t[j] += m < G ? __ldcg(src + (size_t)m * kRedSlots + j) : 0.0;
        }
        fold_quarter<NV>(t, quarter, w);
    }
    __syncthreads();
    if (w == 0) add_quarters<NV>(out, quarter);
}

// init + row sum of lane's row in slice t (all 32 lanes of the warp call it),
// one accumulator: seven warps per SM sub-partition keep its FP64 pipe busy,
// so the chain's latency is hidden, and starting from init (beta q in the
// iteration) saves the separate add of the recurrence.  x is written by this
// kernel between grid barriers, so its loads are plain coherent loads
// (L1-cached: the acquire fence of every grid barrier drops stale L1 lines),
// never the read-only path; the matrix goes through L2 only, leaving L1 to
// the gathered window of x.
// Entries k0 <= k < k1 of the slice (k1 < 0: to the slice width), in
// batches of U entries (all loads of a batch in flight before its FMAs),
// then of kSellUnroll, then one at a time.
// sell_slice_sum_at takes the slice's first entry a and its width wt (a
// caller that keeps them saves the two dependent loads of M.ptr per call).
template <int U = kSellUnroll>
__device__ __forceinline__ double sell_slice_sum_at(const SellMatrix &M, int t, long long a, int wt, const double *x,
                                                    double init, int k0 = 0, int k1 = -1) {
    const int lane = threadIdx.x & 31;
    const bool st = M.stream != 0;
    const int w = k1 >= 0 ? k1 : wt;
    const int row = t * 32 + lane;
    const double *vv = M.vals + a + lane;
    double s = init;
    int k = k0;
    if (M.cols16) {
        const int16_t *cc = M.cols16 + a + lane;
        if constexpr (U != kSellUnroll) {
            for (; k + U <= w; k += U) {
                double vr[U], xr[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    vr[u] = mload(vv + (k + u) * 32, st);
                    xr[u] = __ldca(x + bchk(row + (int)mload(cc + (k + u) * 32, st), M.n));
                }
#pragma unroll
                for (int u = 0; u < U; ++u) s = fma(vr[u], xr[u], s);
            }
        }
        for (; k + kSellUnroll <= w; k += kSellUnroll) {
            double vr[kSellUnroll], xr[kSellUnroll];
#pragma unroll
            for (int u = 0; u < kSellUnroll; ++u) {
                vr[u] = mload(vv + (k + u) * 32, st);
                xr[u] = __ldca(x + bchk(row + (int)mload(cc + (k + u) * 32, st), M.n));
            }
#pragma unroll
            for (int u = 0; u < kSellUnroll; ++u) s = fma(vr[u], xr[u], s);
        }
        for (; k < w; ++k) s = fma(mload(vv + k * 32, st), __ldca(x + bchk(row + (int)mload(cc + k * 32, st), M.n)), s);
    } else {
        const int32_t *cc = M.cols32 + a + lane;
        if constexpr (U != kSellUnroll) {
            for (; k + U <= w; k += U) {
                double vr[U], xr[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    vr[u] = mload(vv + (k + u) * 32, st);
                    xr[u] = __ldca(x + bchk(mload(cc + (k + u) * 32, st), M.n));
                }
#pragma unroll
                for (int u = 0; u < U; ++u) s = fma(vr[u], xr[u], s);
            }
        }
        for (; k + kSellUnroll <= w; k += kSellUnroll) {
            double vr[kSellUnroll], xr[kSellUnroll];
#pragma unroll
            for (int u = 0; u < kSellUnroll; ++u) {
                vr[u] = mload(vv + (k + u) * 32, st);
                xr[u] = __ldca(x + bchk(mload(cc + (k + u) * 32, st), M.n));
            }
#pragma unroll
            for (int u = 0; u < kSellUnroll; ++u) s = fma(vr[u], xr[u], s);
        }
        for (; k < w; ++k) s = fma(mload(vv + k * 32, st), __ldca(x + bchk(mload(cc + k * 32, st), M.n)), s);
    }
    return s;
}

template <int U = kSellUnroll>
__device__ __forceinline__ double sell_slice_sum(const SellMatrix &M, int t, const double *x, double init,
                                                 int k0 = 0, int k1 = -1) {
    const long long a = M.ptr[t];
    return sell_slice_sum_at<U>(M, t, a, (int)((M.ptr[t + 1] - a) >> 5), x, init, k0, k1);
}

}  // namespace gbcg
