// SpMV in the SELL-32 layout, read straight from global memory (sm_103a).
//
// Slice t holds rows 32t .. 32t+31 padded to the longest of them (w_t
// entries); entry k of lane l sits at offset slice_ptr[t] + 32 k + l, so the
// warp that owns a slice reads 32 consecutive values, 32 consecutive
// columns and, for a stencil (the k-th neighbour of consecutive rows is at
// a constant offset), 32 consecutive entries of x per step: every load is
// coalesced, nothing is staged in shared memory, and any number of warps
// can run per SM.  Columns are 16-bit offsets from the row (cols16) when
// every |col - row| < 2^15, else 32-bit column indices (cols32).  Padded
// entries have value 0 and point at the row itself.
//
// Exactly one FMA per stored entry (plus padding, below 1% for Q1 boxes);
// the summation order differs from the tiled kernels only in association.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "check.cuh"

namespace gbcg {

struct SellMatrix {
    int32_t n;
    int32_t nslices;
    int32_t stream;                        // 1: matrix loads marked evict-first (matrix larger than L2)
    const long long *__restrict__ ptr;     // nslices + 1 entry offsets (multiples of 32)
    const double *__restrict__ vals;       // padded entries
    const int16_t *__restrict__ cols16;    // col - row, or nullptr
    const int32_t *__restrict__ cols32;    // col, when cols16 is nullptr
    const int32_t *__restrict__ split;     // per slice: width of the block of entries in the CTA's own
                                           // rows (slice solve kernel layout), or nullptr
};

constexpr int kSellThreads = 256;
constexpr int kSellBlocksPerSm = 8;
constexpr int kSellUnroll = 9;

// Matrix loads: streaming (evict-first, read once per SpMV) when the matrix
// does not fit L2, plain (kept in L2 across SpMVs) when it does.
template <class T>
__device__ __forceinline__ T mload(const T *p, bool stream) {
    return stream ? __ldcs(p) : __ldcg(p);
}

// Row sums of the slices owned by this warp (grid-stride over slices):
// epi.row(i, sum) for every row i < n.
template <class Epi>
__device__ __forceinline__ void sell_rows(const SellMatrix &M, const double *__restrict__ x, Epi &epi) {
    const bool st = M.stream != 0;
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int t = warp; t < M.nslices; t += nwarps) {
        const long long a = M.ptr[t];
        const int w = (int)((M.ptr[t + 1] - a) >> 5);
        const int row = t * 32 + lane;
        const double *vv = M.vals + a + lane;
        double s0 = 0.0, s1 = 0.0;
        int k = 0;
        if (M.cols16) {
            const int16_t *cc = M.cols16 + a + lane;
            for (; k + kSellUnroll <= w; k += kSellUnroll) {
                double vr[kSellUnroll], xr[kSellUnroll];
#pragma unroll
                for (int u = 0; u < kSellUnroll; ++u) {
                    vr[u] = mload(vv + (k + u) * 32, st);
                    xr[u] = __ldg(x + bchk(row + (int)mload(cc + (k + u) * 32, st), M.n));
                }
#pragma unroll
                for (int u = 0; u < kSellUnroll; ++u) {
                    if (u & 1) s1 = fma(vr[u], xr[u], s1);
                    else s0 = fma(vr[u], xr[u], s0);
                }
            }
            for (; k < w; ++k) s0 = fma(mload(vv + k * 32, st), __ldg(x + bchk(row + (int)mload(cc + k * 32, st), M.n)), s0);
        } else {
            const int32_t *cc = M.cols32 + a + lane;
            for (; k + kSellUnroll <= w; k += kSellUnroll) {
                double vr[kSellUnroll], xr[kSellUnroll];
#pragma unroll
                for (int u = 0; u < kSellUnroll; ++u) {
                    vr[u] = mload(vv + (k + u) * 32, st);
                    xr[u] = __ldg(x + bchk(mload(cc + (k + u) * 32, st), M.n));
                }
#pragma unroll
                for (int u = 0; u < kSellUnroll; ++u) {
                    if (u & 1) s1 = fma(vr[u], xr[u], s1);
                    else s0 = fma(vr[u], xr[u], s0);
                }
            }
            for (; k < w; ++k) s0 = fma(mload(vv + k * 32, st), __ldg(x + bchk(mload(cc + k * 32, st), M.n)), s0);
        }
        if (row < M.n) epi.row(row, s0 + s1, 0);
    }
}

}  // namespace gbcg
