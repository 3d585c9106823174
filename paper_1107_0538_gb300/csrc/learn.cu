// Learned preconditioner for CG on Q1 node grids, flexible CG around it, and
// the kernels that train it (sm_103a).
//
// The paper (Section IV) runs unpreconditioned CG; this file adds the
// preconditioner z = D^-1/2 L^T L D^-1/2 r, L = C2 diag(g) C1, a
// convolutional network over the node grid (C1: 1 -> 16 channels, C2:
// 16 -> 16, 3x3x3 taps, gates g from log nu).  Everything the network touches
// lives in a zero-padded node grid, channels last:
//
//   padded node (x+1, y+1, z+1), x fastest, (nx+2)(ny+2)(nz+2) positions plus
//   a zero tail; a 16-channel BF16 activation is 32 bytes per position.
//
// The convolutions take BF16 inputs and accumulate in FP32.  The training
// convolutions and C1 are implicit GEMMs on mma.sync m16n8k16: a CTA (8
// warps) computes a brick of 16 x 8 x 4 output nodes; an M-tile is one x-row
// of the brick (16 consecutive nodes), so each of the 27 taps reads 16
// consecutive rows of the staged input (a constant shift).  The brick's
// input with its one-node halo (18 x 10 x 6 positions, 35 KB for 16
// channels) is staged once into shared memory with a bank-conflict-free
// swizzle of the two 16-byte halves of each row; outputs past the grid
// (ragged bricks) are computed and dropped, so every store goes to an
// interior node and the zero halo is never overwritten.  The solve's 16 -> 16
// convolutions run on tcgen05 (conv16tc_kernel) and its 16 -> 1 convolution
// on the FP32 pipe (convout_kernel).
//
// Flexible CG runs as a CUDA graph of kUnroll iterations of five kernels
// (conv C1, conv C2, conv C2^T, conv C1^T + z + dots, and one cooperative
// kernel for the SpMV of z with the p = z + beta p and q = A z + beta q
// updates, p.q, the x, r update and the stop test); handles without SELL-32
// CTA ranges run the last as two kernels (the tiled SpMV, then the x, r
// update).  Scalars are decided by the last CTA to finish each reducing
// kernel, or by every CTA after the grid barrier (fixed-order sums: bitwise
// reproducible), and kept in a device state block; kernels return at once
// after the solve is done.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <new>
#include <type_traits>
#include <vector>

#include "cg_device.cuh"
#include "gbcg.h"
#include "handle.h"
#include "lowprec.h"
#include "sellsolve.cuh"

using namespace gbcg;

namespace {

constexpr int kCh = 16, kTaps = 27, kTapsPad = 32, kCentre = 13;
constexpr int kOffW1 = 0, kOffW2 = kCh * kTaps, kOffWg = kOffW2 + kCh * kCh * kTaps, kOffBg = kOffWg + kCh * kTaps;
static_assert(kOffBg + kCh == CG_LEARN_PARAMS, "parameter layout");
constexpr float kLogNuScale = 0.125f;

constexpr int kBX = 16, kBY = 8, kBZ = 4;                 // output brick of a conv CTA
constexpr int kSX = kBX + 2, kSY = kBY + 2, kSZ = kBZ + 2;   // staged brick with its halo
constexpr int kStaged = kSX * kSY * kSZ;                     // 1080 positions
constexpr int kRows = kBY * kBZ;                             // M-tiles (x-rows) per brick
constexpr int kCT = 256;                                     // threads of a conv CTA (8 warps)
constexpr int kMTiles = kRows / (kCT / 32);                  // M-tiles per warp
constexpr int kSlack = 64;       // zero positions after the padded grid
constexpr int kVT = 256;         // threads of the vector kernels
constexpr int kMaxWindow = 128;
constexpr int kUnroll = 6;       // iterations per graph launch
static_assert(kMTiles == 4, "warp w owns rows 4 (w & 1) .. + 3 of plane w / 2");

constexpr int kModeLearned = 0, kModeJacobi = 1;

// ----------------------------------------------------------------- geometry
struct Geo {
    int nx, ny, nz;       // nodes per axis
    int px, py, pz;       // padded extents
    int plane;            // px * py
    int bx, by, bz, tiles;
    int tbx, tby, tbz, ttiles;   // bricks of the tensor-core 16 -> 16 convolution
    int n;                // nodes
    long long npad;       // px py pz
};

Geo make_geo(int ex, int ey, int ez) {
    Geo G{};
    G.nx = ex + 1;
    G.ny = ey + 1;
    G.nz = ez + 1;
    G.px = G.nx + 2;
    G.py = G.ny + 2;
    G.pz = G.nz + 2;
    G.plane = G.px * G.py;
    G.bx = (G.nx + kBX - 1) / kBX;
    G.by = (G.ny + kBY - 1) / kBY;
    G.bz = (G.nz + kBZ - 1) / kBZ;
    G.tiles = G.bx * G.by * G.bz;
    G.tbx = (G.nx + 7) / 8;
    G.tby = (G.ny + 15) / 16;
    G.tbz = (G.nz + 3) / 4;
    G.ttiles = G.tbx * G.tby * G.tbz;
    G.n = G.nx * G.ny * G.nz;
    G.npad = (long long)G.px * G.py * G.pz;
    return G;
}

constexpr size_t kStage16 = (size_t)kStaged * 32;
constexpr size_t kStage1 = ((size_t)kStaged * 2 + 15) / 16 * 16;
constexpr size_t kDyTile = (size_t)kBX * kRows * 32;
size_t conv16_smem(const Geo &) { return kStage16 + (size_t)kTaps * kCh * kCh * 2; }
size_t conv1_smem(const Geo &) { return kStage1; }
// the 16 -> 1 convolution stages its input rows 32 bytes apart more: a row
// is 152 words, 24 mod 32, so 4 consecutive rows start 8 banks apart
constexpr int kOutRowBytes = kSX * 32 + 32;
static_assert(kOutRowBytes % 16 == 0, "16-byte aligned staged rows");
constexpr size_t kOutStage = (size_t)kSY * kSZ * kOutRowBytes;   // one staged brick
size_t convout_smem(const Geo &) { return 2 * kOutStage; }          // two: the next brick loads meanwhile
size_t wgrad16_smem(const Geo &) { return kStage16 + kDyTile; }
size_t wgrad1_smem(const Geo &) { return kStage1 + kDyTile + (size_t)(kCT / 32) * 16 * 32 * 4; }

// ---------------------------------------------------------------- device
__device__ __forceinline__ int tap_dx(int t) { return t % 3 - 1; }
__device__ __forceinline__ int tap_dy(int t) { return (t / 3) % 3 - 1; }
__device__ __forceinline__ int tap_dz(int t) { return t / 9 - 1; }

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }


__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}
// D += A B, m16n8k16, A row-major 16x16 BF16, B column-major 16x8 BF16, FP32.
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}
__device__ __forceinline__ float2 unpack_bf16(uint32_t u) {
    __nv_bfloat162 v = *reinterpret_cast<__nv_bfloat162 *>(&u);
    return __bfloat1622float2(v);
}
__device__ __forceinline__ uint32_t pack_raw(uint16_t lo, uint16_t hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }

// Row R (32 bytes: two 16-byte halves) of a swizzled staging buffer: half h
// lives at (h ^ bit 2 of R), so 8 consecutive rows hit 8 distinct bank groups.
__device__ __forceinline__ uint32_t row_addr(uint32_t base, int R, int h) {
    return base + (uint32_t)R * 32u + ((uint32_t)(h ^ ((R >> 2) & 1)) << 4);
}

// A brick: origin (x0, y0, z0) of its outputs in node coordinates.
struct Brick {
    int x0, y0, z0;
};
__device__ __forceinline__ Brick brick_of(const Geo &G, int tile) {
    const int tx = tile % G.bx, rest = tile / G.bx;
    return Brick{tx * kBX, (rest % G.by) * kBY, (rest / G.by) * kBZ};
}

// Staged position (xs, ys, zs) of a brick is padded node (x0 + xs, y0 + ys,
// z0 + zs); its row (ys, zs) exists in the padded grid when
// y0 + ys < py and z0 + zs < pz (rows past it only feed dropped outputs).
__device__ __forceinline__ bool staged_row(const Geo &G, const Brick &B, int ys, int zs, long long &pos0) {
    const int py = B.y0 + ys, pz = B.z0 + zs;
    pos0 = (long long)pz * G.plane + (long long)py * G.px + B.x0;
    return py < G.py && pz < G.pz;
}

// Stages the 16-channel input of a brick (rows of 18 positions, 36 chunks of 16 bytes).
__device__ __forceinline__ void stage16(const Geo &G, const Brick &B, const __nv_bfloat16 *src, unsigned char *sm) {
    constexpr int kChunks = kSX * 2;
    for (int c = threadIdx.x; c < kSY * kSZ * kChunks; c += blockDim.x) {
        const int row = c / kChunks, k = c - row * kChunks;
        const int xs = k >> 1, h = k & 1;
        const int ys = row % kSY, zs = row / kSY;
        const int R = row * kSX + xs;
        unsigned char *dst = sm + R * 32 + ((h ^ ((R >> 2) & 1)) << 4);
        long long pos0;
        if (staged_row(G, B, ys, zs, pos0)) cp_async16(dst, src + (pos0 + xs) * kCh + h * 8);
        else *reinterpret_cast<uint4 *>(dst) = make_uint4(0u, 0u, 0u, 0u);
    }
}

// One-channel input of a brick (a padded BF16 field).
__device__ __forceinline__ void stage1(const Geo &G, const Brick &B, const __nv_bfloat16 *src, uint16_t *sm) {
    for (int c = threadIdx.x; c < kStaged; c += blockDim.x) {
        const int row = c / kSX, xs = c - row * kSX;
        const int ys = row % kSY, zs = row / kSY;
        long long pos0;
        sm[c] = staged_row(G, B, ys, zs, pos0) ? reinterpret_cast<const uint16_t *>(src)[pos0 + xs] : (uint16_t)0;
    }
}

// Output row r of a warp's M-tile m: node coordinates and validity.
struct OutRow {
    int x, y, z;
    bool ok;
};
__device__ __forceinline__ OutRow out_row(const Geo &G, const Brick &B, int w, int m, int r) {
    OutRow o{B.x0 + r, B.y0 + 4 * (w & 1) + m, B.z0 + (w >> 1), false};
    o.ok = o.x < G.nx && o.y < G.ny && o.z < G.nz;
    return o;
}
__device__ __forceinline__ long long padded_pos(const Geo &G, int x, int y, int z) {
    return (long long)(z + 1) * G.plane + (long long)(y + 1) * G.px + (x + 1);
}
// Staged row index of the A operand of warp w, M-tile m, for tap offsets (dx, dy, dz).
__device__ __forceinline__ int a_row(int w, int m, int dx, int dy, int dz) {
    return (((w >> 1) + 1 + dz) * kSY + (4 * (w & 1) + m + 1 + dy)) * kSX + 1 + dx;
}

// ------------------------------------------------------- solver state
struct FcgState {
    const double *b;
    double *x;
    double tol, bnorm, bb;
    double rho, alpha, beta, rr, rdr, sigma, sigma_inv, zr, zq, pq, true_rr;
    double best_before, factor;
    double ring[kMaxWindow + 1];
    int32_t n, iters, status, done, mode, restart, reverted_at, mode_start, maxit, window;
    unsigned int counter;
    unsigned int bar_count, bar_gen;   // grid barrier of the fused SELL-32 kernel (resets itself)
    int32_t pad;
};

// Flags the host polls after each graph launch (the same order as in FcgState).
struct FcgFlags {
    int32_t n, iters, status, done, mode;
};

struct ConvArgs {
    Geo G;
    const __nv_bfloat16 *in;     // padded input (16 channels, or 1 channel for conv1)
    const double *dsq;           // 1 / sqrt(diag A)
    const float *dsq32;          // the same in FP32 (E_OUT_Z, E_OUT_FCG: z = sigma D^-1/2 u in FP32)
    const __nv_bfloat16 *w;      // packed weights of this convolution
    const float *bias;           // E_SIGMOID
    __nv_bfloat16 *out;          // padded 16-channel output
    __nv_bfloat16 *pre;          // E_GATE_PRE: pre-gate output; E_BWD_GATE: pre-gate field read
    const __nv_bfloat16 *gate;   // gates (padded, 16 channels)
    float *dg;                   // E_BWD_GATE: gate-gradient field (padded, 16 channels, FP32)
    int dg_add;                  // 0: dg = ..., 1: dg += ...
    // conv_out
    float *u;                    // E_OUT_U: node-order FP32 output
    double *z;                   // E_OUT_Z / E_OUT_FCG
    const double *r;             // E_OUT_FCG: residual (node order)
    const double *q;             // E_OUT_FCG: A p of the last step
    const double *dinv;          // Jacobi fallback
    double *partials;
    FcgState *st;                // solver state (nullptr: always run; conv1 scales by sigma[1] if set)
    const double *sigma;         // apply: {sigma, 1/sigma}: conv1 output scale, conv_out output scale
    unsigned long long wait_ns;  // bound of the tensor-core kernel's wait for its MMAs
    int *err;                    // that kernel's timeout report when st is nullptr (or nullptr)
};

enum { E_STORE = 0, E_GATE = 1, E_GATE_PRE = 2, E_BWD_GATE = 3, E_SIGMOID = 4 };
enum { E_OUT_U = 0, E_OUT_Z = 1, E_OUT_FCG = 2 };

__device__ __forceinline__ bool conv_skip(const FcgState *st) {
    return st && (st->done || st->mode != kModeLearned);
}

// Gates of a warp's output rows, loaded ahead of the MMA loop: gv[m][hrow][nb]
// (two channels each), zero for dropped rows.
template <int EPI>
__device__ __forceinline__ void load_gates(const ConvArgs &A, const Brick &B, int w,
                                           uint32_t (&gv)[kMTiles][2][2]) {
    if (EPI != E_GATE && EPI != E_GATE_PRE && EPI != E_BWD_GATE) return;
    const int lane = threadIdx.x & 31, g = lane >> 2, t4 = lane & 3;
#pragma unroll
    for (int m = 0; m < kMTiles; ++m)
#pragma unroll
        for (int hrow = 0; hrow < 2; ++hrow) {
            const OutRow o = out_row(A.G, B, w, m, g + 8 * hrow);
            const long long pos = padded_pos(A.G, o.x, o.y, o.z);
#pragma unroll
            for (int nb = 0; nb < 2; ++nb)
                gv[m][hrow][nb] = o.ok ? __ldg(reinterpret_cast<const unsigned int *>(A.gate + pos * kCh + nb * 8 + 2 * t4))
                                       : 0u;
        }
}

// 16-channel output of one warp's M-tiles: acc[m][nb][4] (rows g, g+8;
// columns 2t4, 2t4+1 of n-block nb), scaled by oscale first.
template <int EPI>
__device__ __forceinline__ void store16(const ConvArgs &A, const Brick &B, int w, float (&acc)[kMTiles][2][4],
                                        const uint32_t (&gvv)[kMTiles][2][2], float oscale) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t4 = lane & 3;
#pragma unroll
    for (int m = 0; m < kMTiles; ++m) {
#pragma unroll
        for (int hrow = 0; hrow < 2; ++hrow) {
            const OutRow o = out_row(A.G, B, w, m, g + 8 * hrow);
            if (!o.ok) continue;
            const long long pos = padded_pos(A.G, o.x, o.y, o.z);
#pragma unroll
            for (int nb = 0; nb < 2; ++nb) {
                const int ch = nb * 8 + 2 * t4;
                const long long e = pos * kCh + ch;
                float v0 = acc[m][nb][2 * hrow] * oscale, v1 = acc[m][nb][2 * hrow + 1] * oscale;
                if (EPI == E_SIGMOID) {
                    v0 = 1.0f / (1.0f + __expf(-(v0 + A.bias[ch])));
                    v1 = 1.0f / (1.0f + __expf(-(v1 + A.bias[ch + 1])));
                    *reinterpret_cast<uint32_t *>(A.out + e) = pack_bf16(v0, v1);
                } else if (EPI == E_STORE) {
                    *reinterpret_cast<uint32_t *>(A.out + e) = pack_bf16(v0, v1);
                } else {
                    const float2 gv = unpack_bf16(gvv[m][hrow][nb]);
                    if (EPI == E_GATE_PRE) *reinterpret_cast<uint32_t *>(A.pre + e) = pack_bf16(v0, v1);
                    if (EPI == E_BWD_GATE) {
                        const float2 pv = unpack_bf16(*reinterpret_cast<const uint32_t *>(A.pre + e));
                        float2 *d = reinterpret_cast<float2 *>(A.dg + e);
                        float2 dv = A.dg_add ? *d : make_float2(0.0f, 0.0f);
                        dv.x = fmaf(pv.x, v0, dv.x);
                        dv.y = fmaf(pv.y, v1, dv.y);
                        *d = dv;
                    }
                    *reinterpret_cast<uint32_t *>(A.out + e) = pack_bf16(gv.x * v0, gv.y * v1);
                }
            }
        }
    }
}

// ------------------------------------------------- 16 -> 16 convolution
// y[o, p] = sum_{t, c} K[t][o][c] x[c, p + off(t)], K packed [27][16][16].
template <int EPI>
__global__ void __launch_bounds__(kCT, 3) conv16_kernel(ConvArgs A) {
    if (conv_skip(A.st)) return;
    extern __shared__ __align__(128) unsigned char sm[];
    const Geo &G = A.G;
    unsigned char *sw = sm + kStage16;
    const Brick B = brick_of(G, blockIdx.x);
    stage16(G, B, A.in, sm);
    const int w = threadIdx.x >> 5;
    uint32_t gv[kMTiles][2][2];
    load_gates<EPI>(A, B, w, gv);
    // weights: row (t, o) of 32 bytes, swizzled like the input
    for (int idx = threadIdx.x; idx < kTaps * kCh * 2; idx += blockDim.x) {
        const int R = idx >> 1, h = idx & 1;
        cp_async16(sw + R * 32 + ((h ^ ((R >> 2) & 1)) << 4), A.w + (size_t)R * kCh + h * 8);
    }
    cp_async_wait_all();
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint32_t in_base = smem_u32(sm), w_base = smem_u32(sw);
    float acc[kMTiles][2][4];
#pragma unroll
    for (int m = 0; m < kMTiles; ++m)
#pragma unroll
        for (int nb = 0; nb < 2; ++nb)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[m][nb][k] = 0.0f;
    const int a_r = (lane & 7) + ((lane >> 3) & 1) * 8, a_half = lane >> 4;
    const int b_o = (lane & 7) + ((lane >> 4) << 3), b_half = (lane >> 3) & 1;
#pragma unroll
    for (int t = 0; t < kTaps; ++t) {
        uint32_t b[4];
        ldsm_x4(b, row_addr(w_base, t * kCh + b_o, b_half));
#pragma unroll
        for (int m = 0; m < kMTiles; ++m) {
            uint32_t a[4];
            ldsm_x4(a, row_addr(in_base, a_row(w, m, tap_dx(t), tap_dy(t), tap_dz(t)) + a_r, a_half));
            mma_bf16(acc[m][0], a, b[0], b[1]);
            mma_bf16(acc[m][1], a, b[2], b[3]);
        }
    }
    store16<EPI>(A, B, w, acc, gv, 1.0f);
}

// ------------------------------------ 16 -> 16 convolution on tcgen05
// The convolution of conv16_kernel (E_STORE, E_GATE: the flexible-CG body and
// the stand-alone apply) on the 5th-generation tensor cores.  A CTA owns a
// brick of 8 (x) x 16 (y) x 4 (z) outputs.  Its input with the halo (10 x 18
// x 6 positions) is staged channel-split: channels 0-7 of every position in
// one plane of 16-byte rows, channels 8-15 in a second plane.  The 128
// outputs of a z-plane of the brick (x fastest, 8 per y) then form an
// M = 128 operand in the canonical K-major layout without swizzle: 8-row
// core matrices of consecutive x, 16 bytes per row, y groups one staged row
// (160 bytes) apart, the two K halves one plane apart.  Tap (dx, dy, dz) is
// the same operand moved by dx + 10 dy + 180 dz positions, so each of the 27
// taps is one MMA (M = 128, N = 16, K = 16; BF16 in, FP32 accumulate) into
// the plane's 16 TMEM columns: 108 MMAs per brick, issued by one thread per
// plane, completing on an mbarrier.  Warps w and w + 4 read TMEM lanes
// 32 (w mod 4) .. + 31 (output i = lane index) of alternate planes.
constexpr int kTX = 8, kTY = 16, kTZ = 4;
constexpr int kTSX = kTX + 2, kTSY = kTY + 2, kTSZ = kTZ + 2;
constexpr int kTStaged = kTSX * kTSY * kTSZ;                  // 1080 positions
constexpr uint32_t kTPlane = (uint32_t)kTStaged * 16;          // bytes of one channel half
constexpr uint32_t kTWeights = (uint32_t)kTaps * kCh * kCh * 2;  // 13824 bytes
constexpr uint32_t kTCols = 64;                                // TMEM columns: 4 planes x 16
static_assert(kTX * kTY == 128, "one M = 128 operand per z-plane");
size_t conv16tc_smem(const Geo &) { return 2 * (size_t)kTPlane + kTWeights + 16; }

// Shared-memory matrix descriptor (SM100 version 1), no swizzle: start, LBO
// (K-direction core-matrix stride) and SBO (M/N-direction 8-row group
// stride), each in 16-byte units.
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: FP32 D, BF16 A and B, both K-major,
// N = 16 (bits 17-22: N / 8), M = 128 (bits 24-28: M / 16).
constexpr uint32_t kConvIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// 16 consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void finish(FcgState *st, int status);

template <int EPI>
__global__ void __launch_bounds__(kCT) conv16tc_kernel(ConvArgs A) {
    static_assert(EPI == E_STORE || EPI == E_GATE, "forward epilogues only");
    if (conv_skip(A.st)) return;
    extern __shared__ __align__(128) unsigned char sm[];
    const Geo &G = A.G;
    unsigned char *sw = sm + 2 * kTPlane;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sw + kTWeights);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
    const int tile = blockIdx.x, rest = tile / G.tbx;
    const int x0 = (tile % G.tbx) * kTX, y0 = (rest % G.tby) * kTY, z0 = (rest / G.tby) * kTZ;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // input with halo: staged position (xs, ys, zs) is padded node
    // (x0 + xs, y0 + ys, z0 + zs); rows past the padded grid are zero.  A
    // warp copies one staged row (10 positions: 320 contiguous bytes) at a
    // time, lane l < 20 one 16-byte chunk.
    {
        const int xs = lane >> 1, h = lane & 1;
        for (int row = w; row < kTSY * kTSZ; row += kCT / 32) {
            if (lane >= 2 * kTSX) continue;
            const int ys = row % kTSY, zs = row / kTSY;
            const int py = y0 + ys, pz = z0 + zs;
            unsigned char *dst = sm + h * kTPlane + (uint32_t)(row * kTSX + xs) * 16;
            if (py < G.py && pz < G.pz)
                cp_async16(dst, A.in + ((long long)pz * G.plane + (long long)py * G.px + x0 + xs) * kCh + h * 8);
            else
                *reinterpret_cast<uint4 *>(dst) = make_uint4(0u, 0u, 0u, 0u);
        }
    }
    // weights of tap t: B = K[t] as 16 (N = output) rows of 16 (K = input)
    // channels, K halves 256 bytes apart, 8-row groups 128 bytes apart; a
    // warp copies one tap (32 chunks) at a time
    for (int t = w; t < kTaps; t += kCT / 32) {
        const int o = lane >> 1, h = lane & 1;
        cp_async16(sw + t * 512 + h * 256 + o * 16, A.w + ((size_t)t * kCh + o) * kCh + h * 8);
    }
    if (w == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(kTCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 32) {
        mbar_init(bar, kTZ);   // one commit per issuing warp
        mbar_init_fence();
    }
    // gates of this thread's outputs, loaded while the MMAs run
    uint4 gq[2][2];
    const int i = 32 * (w & 3) + lane;   // output (M row, TMEM lane) of this thread
    const int ox = x0 + (i & 7), oy = y0 + (i >> 3);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int oz = z0 + (w >> 2) + 2 * k;
        const bool ok = ox < G.nx && oy < G.ny && oz < G.nz;
        const long long pos = padded_pos(G, ox, oy, oz);
        if (EPI == E_GATE && ok) {
            gq[k][0] = __ldg(reinterpret_cast<const uint4 *>(A.gate + pos * kCh));
            gq[k][1] = __ldg(reinterpret_cast<const uint4 *>(A.gate + pos * kCh + 8));
        } else {
            gq[k][0] = gq[k][1] = make_uint4(0u, 0u, 0u, 0u);
        }
    }
    cp_async_wait_all();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // staged data -> tensor-core reads
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    // a thread's tcgen05.mma issue takes ~165 cycles however small the MMA,
    // against ~10 cycles of tensor work at N = 16: lane 0 of warps 0-3 issue
    // the 27 taps of one z-plane each, into their own TMEM columns
    if (lane == 0 && w < kTZ) {
        const int pl = w;
        const uint32_t in_base = smem_u32(sm), w_base = smem_u32(sw);
#pragma unroll 1
        for (int t = 0; t < kTaps; ++t) {
            const int s0 = (1 + tap_dx(t)) + kTSX * ((1 + tap_dy(t)) + kTSY * (1 + pl + tap_dz(t)));
            const uint64_t ad = umma_desc(in_base + (uint32_t)s0 * 16, kTPlane, kTSX * 16);
            const uint64_t bd = umma_desc(w_base + (uint32_t)t * 512, 256, 128);
            umma_bf16(tmem + (uint32_t)pl * 16, ad, bd, kConvIdesc, t > 0 ? 1u : 0u);
        }
        umma_commit(bar);
    }
    bool done = mbar_wait_bounded(bar, 0, A.wait_ns);
    tc_fence_after();
    if (done) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int pl = (w >> 2) + 2 * k;
            uint32_t v[16];
            tmem_ld16(tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)pl * 16, v);
            const int oz = z0 + pl;
            if (ox < G.nx && oy < G.ny && oz < G.nz) {
                const long long pos = padded_pos(G, ox, oy, oz);
                uint32_t o[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    float a0 = __uint_as_float(v[2 * j]), a1 = __uint_as_float(v[2 * j + 1]);
                    if (EPI == E_GATE) {
                        const uint32_t gw = (&gq[k][j >> 2].x)[j & 3];
                        const float2 g = unpack_bf16(gw);
                        a0 *= g.x;
                        a1 *= g.y;
                    }
                    o[j] = pack_bf16(a0, a1);
                }
                uint4 *dst = reinterpret_cast<uint4 *>(A.out + pos * kCh);
                dst[0] = make_uint4(o[0], o[1], o[2], o[3]);
                dst[1] = make_uint4(o[4], o[5], o[6], o[7]);
            }
        }
    } else {
        // report, then give the MMAs in flight a second bounded wait before
        // the columns are freed
        if (threadIdx.x == 0) {
            if (A.st) finish(A.st, CG_ETIMEOUT);
            if (A.err) atomicExch(A.err, CG_ETIMEOUT);
        }
        done = mbar_wait_bounded(bar, 0, A.wait_ns);
    }
    tc_fence_before();
    __syncthreads();
    if (w == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTCols) : "memory");
    }
}

// --------------------------------------------------- 1 -> 16 convolution
// y[o, p] = sum_t K[o][t] x[p + off(t)], K packed [16][32] (taps 27..31 zero):
// the taps are the GEMM's K dimension, gathered from the staged plane.
template <int EPI>
__global__ void __launch_bounds__(kCT) conv1_kernel(ConvArgs A) {
    if (conv_skip(A.st)) return;
    extern __shared__ __align__(128) unsigned char sm[];
    const Geo &G = A.G;
    uint16_t *xs = reinterpret_cast<uint16_t *>(sm);
    const Brick B = brick_of(G, blockIdx.x);
    // the input is D^-1/2 r (flexible CG, apply): scale the output by 1/sigma
    const float oscale = A.st ? (float)A.st->sigma_inv : (A.sigma ? (float)A.sigma[1] : 1.0f);
    stage1(G, B, A.in, xs);
    uint32_t gv[kMTiles][2][2];
    load_gates<EPI>(A, B, threadIdx.x >> 5, gv);
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, g = lane >> 2, t4 = lane & 3;
    // B fragments (whole K = 32 taps): b[ks][nb][2]
    uint32_t b[2][2][2];
    const uint32_t *wk = reinterpret_cast<const uint32_t *>(A.w);
#pragma unroll
    for (int ks = 0; ks < 2; ++ks)
#pragma unroll
        for (int nb = 0; nb < 2; ++nb) {
            const int o = nb * 8 + g;
            b[ks][nb][0] = __ldg(wk + ((o * kTapsPad + ks * 16 + 2 * t4) >> 1));
            b[ks][nb][1] = __ldg(wk + ((o * kTapsPad + ks * 16 + 8 + 2 * t4) >> 1));
        }
    // staged offsets of the taps this lane gathers: k = ks*16 + {2t4, 2t4+1, 2t4+8, 2t4+9}
    int off[2][4];
    bool live[2][4];
#pragma unroll
    for (int ks = 0; ks < 2; ++ks)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int t = ks * 16 + 2 * t4 + (u & 1) + (u >> 1) * 8;
            live[ks][u] = t < kTaps;
            const int tt = t < kTaps ? t : kCentre;
            off[ks][u] = a_row(w, 0, tap_dx(tt), tap_dy(tt), tap_dz(tt));
        }
    float acc[kMTiles][2][4];
#pragma unroll
    for (int m = 0; m < kMTiles; ++m) {
#pragma unroll
        for (int nb = 0; nb < 2; ++nb)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[m][nb][k] = 0.0f;
        const int base = m * kSX + g;   // M-tile m is the next staged row
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            uint16_t v[2][4];
#pragma unroll
            for (int hr = 0; hr < 2; ++hr)
#pragma unroll
                for (int u = 0; u < 4; ++u) v[hr][u] = live[ks][u] ? xs[base + 8 * hr + off[ks][u]] : 0;
            uint32_t a[4];
            a[0] = pack_raw(v[0][0], v[0][1]);
            a[1] = pack_raw(v[1][0], v[1][1]);
            a[2] = pack_raw(v[0][2], v[0][3]);
            a[3] = pack_raw(v[1][2], v[1][3]);
            mma_bf16(acc[m][0], a, b[ks][0][0], b[ks][0][1]);
            mma_bf16(acc[m][1], a, b[ks][1][0], b[ks][1][1]);
        }
    }
    store16<EPI>(A, B, w, acc, gv, oscale);
}

// ----------------------------------------------- deterministic reductions
template <int NV>
__device__ __forceinline__ void cta_sum(double (&v)[NV], double *sred) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        v[j] = warp_sum(v[j]);
        if (lane == 0) sred[j * 32 + w] = v[j];
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) v[j] = warp_sum(lane < nw ? sred[j * 32 + lane] : 0.0);
    }
    __syncthreads();
}

// Sums two values over a CTA of 256 threads and gives the totals to every
// thread.  The values are parked in shared memory (`park`, 512 doubles) and
// value j is added by warp j, 8 entries per lane as a depth-3 tree and then a
// butterfly: the FP64 adds (64 cycles of an SM sub-partition per warp
// instruction on GB300) run on two warps instead of all eight.  Fixed order.
__device__ __forceinline__ void cta_sum2_256(double (&v)[2], double *park, double *sred) {
    park[threadIdx.x] = v[0];
    park[256 + threadIdx.x] = v[1];
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w < 2) {
        const double *q = park + 256 * w + lane;
        double t = ((q[0] + q[32]) + (q[64] + q[96])) + ((q[128] + q[160]) + (q[192] + q[224]));
        t = warp_sum(t);
        if (lane == 0) sred[w] = t;
    }
    __syncthreads();
    v[0] = sred[0];
    v[1] = sred[1];
}

// Publishes this CTA's partials (thread 0 holds them); true in every thread
// of the last CTA to arrive, which then sums all partials into tot (warp 0)
// and resets the counter.  Every thread of that CTA adds a fixed strided
// subset (loads in flight together), then cta_sum combines them: a fixed
// order for a given grid, so the totals are reproducible.
template <int NV>
__device__ __forceinline__ bool last_cta_totals(double (&v)[NV], double *partials, unsigned int *counter,
                                                double (&tot)[NV], int *sflag, double *sred) {
    if (threadIdx.x == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) partials[(size_t)j * gridDim.x + blockIdx.x] = v[j];
        __threadfence();
        *sflag = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!*sflag) return false;
    __threadfence();
    const int G = (int)gridDim.x;
    double acc[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) acc[j] = 0.0;
#pragma unroll 4
    for (int m = threadIdx.x; m < G; m += blockDim.x) {
#pragma unroll
        for (int j = 0; j < NV; ++j) acc[j] += __ldcg(partials + (size_t)j * G + m);
    }
    cta_sum<NV>(acc, sred);
#pragma unroll
    for (int j = 0; j < NV; ++j) tot[j] = acc[j];
    if (threadIdx.x == 0) *counter = 0u;
    return true;
}

__device__ __forceinline__ void finish(FcgState *st, int status) {
    st->status = status;
    st->done = 1;
}

// ------------------------------------------------ 16 -> 1 convolution
// u[p] = sum_{t, c} K[t][c] x[c, p + off(t)] (K packed [27][16]).  EPI:
// E_OUT_U stores u (FP32, node order), E_OUT_Z stores z = sigma D^-1/2 u,
// E_OUT_FCG also forms z.r and z.q and takes the flexible-CG decisions (in
// the Jacobi fallback it forms z = D^-1 r instead of running the network).
//
// With one output channel this is 432 multiply-adds per node, and as a
// tensor-core GEMM each output would need its own 27 A fragments (864 bytes
// of shared memory) for one real column of the product.  So it runs on the
// FP32 pipe (packed f32x2 FMAs, two channels an instruction),
// register-blocked: the 4 lanes of a quad split the 16 input channels (4
// each) and own 8 consecutive x outputs of one brick row, and
// for each (dy, dz) they walk the 10 staged positions of the input row once:
// every loaded input feeds up to three outputs (dx = -1, 0, 1) from
// registers.  The quad then adds its four channel partials (a butterfly:
// the same bits in every lane).  Input rows are staged 608 bytes apart (18
// positions of 32 bytes plus 32), so the 32-byte pieces of the 4 rows a warp
// reads at once fall on disjoint groups of 8 banks: a warp's load takes the
// minimum two wavefronts (the shared-memory pipe bounds this kernel).  The kernel is persistent: a CTA loops over its share of
// the bricks with two staging buffers, so the copies of the next brick run
// while the current one is multiplied, the weights are read once per CTA and
// each CTA publishes one partial of z.r and z.q.
// Stages a brick's 16-channel input rows with the TMA unit: one 1-D bulk
// copy per staged row (18 positions, 576 contiguous bytes of the padded
// grid), completing on bar.  Thread r < kSY kSZ issues row r (or zero-fills
// it when the row lies past the padded grid); thread 0 also arrives on bar
// with the bytes expected.  The proxy fence orders the buffer's earlier
// reads and plain stores before the copy overwrites it.
__device__ __forceinline__ void stage16_rows_tma(const Geo &G, const Brick &B, const __nv_bfloat16 *src,
                                                 unsigned char *sm, uint64_t *bar) {
    const int ly = max(0, min(kSY, G.py - B.y0)), lz = max(0, min(kSZ, G.pz - B.z0));   // live rows per axis
    if (threadIdx.x == 0) mbar_arrive_expect_tx(bar, (uint32_t)(ly * lz * kSX * 32));
    const int r = threadIdx.x;
    if (r < kSY * kSZ) {
        const int ys = r % kSY, zs = r / kSY;
        unsigned char *dst = sm + r * kOutRowBytes;
        long long pos0;
        if (staged_row(G, B, ys, zs, pos0)) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tma_load_1d(dst, src + pos0 * kCh, kSX * 32, bar, false);
        } else {
            for (int c = 0; c < kSX * 2; ++c) reinterpret_cast<uint4 *>(dst)[c] = make_uint4(0u, 0u, 0u, 0u);
        }
    }
}

__device__ __forceinline__ float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }
// Two BF16 values (low, high half) as two FP32 values in one 64-bit register
// pair, and the packed FP32 FMA d = a * b + c on such pairs (two IEEE
// round-to-nearest FMAs in one instruction).
__device__ __forceinline__ uint64_t bf16x2_f32x2(uint32_t v) {
    uint64_t d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "r"(v << 16), "r"(v & 0xffff0000u));
    return d;
}
__device__ __forceinline__ uint64_t ffma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// A lane's two output nodes x, x + 1 of a brick row (node index i0 of the
// first) and the epilogue operands the 16 -> 1 convolution needs for them;
// nodes past the grid (or no brick: live = false) load nothing and get zeros.
struct OutNodes {
    int i0;
    bool ok0, ok1;
    float d0, d1;
    double r0, r1, q0, q1;
};
template <int EPI>
__device__ __forceinline__ OutNodes out_nodes(const ConvArgs &A, const Brick &B, int xh, int oy, int oz, int j4,
                                              bool live) {
    const Geo &G = A.G;
    OutNodes o{};
    const int ox = B.x0 + xh * 8 + 2 * j4, gy = B.y0 + oy, gz = B.z0 + oz;
    const bool rowok = live && gy < G.ny && gz < G.nz;
    o.ok0 = rowok && ox < G.nx;
    o.ok1 = rowok && ox + 1 < G.nx;
    o.i0 = ox + G.nx * (gy + G.ny * gz);
    if (EPI != E_OUT_U) {
        if (o.ok0) o.d0 = __ldg(A.dsq32 + o.i0);
        if (o.ok1) o.d1 = __ldg(A.dsq32 + o.i0 + 1);
    }
    if (EPI == E_OUT_FCG) {
        if (o.ok0) {
            o.r0 = __ldcg(A.r + o.i0);
            o.q0 = __ldcg(A.q + o.i0);
        }
        if (o.ok1) {
            o.r1 = __ldcg(A.r + o.i0 + 1);
            o.q1 = __ldcg(A.q + o.i0 + 1);
        }
    }
    return o;
}

template <int EPI>
__global__ void __launch_bounds__(kCT) convout_kernel(ConvArgs A) {
    FcgState *st = A.st;
    if (st && st->done) return;
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ double sred[2 * 32];
    __shared__ float4 swt[kTaps * 4];   // tap t, channels 4 j .. 4 j + 3 at swt[4 t + j]
    __shared__ __align__(8) uint64_t sbar[2];   // TMA completion of the two staging buffers
    __shared__ int sflag, sswitch;
    const Geo &G = A.G;
    const bool learned = !st || st->mode == kModeLearned;
    double dzr = 0.0, dzq = 0.0;
    if (learned) {
        if (threadIdx.x < kTaps * 4) {
            const uint2 v = __ldg(reinterpret_cast<const uint2 *>(A.w) + threadIdx.x);   // 4 BF16 weights
            swt[threadIdx.x] = make_float4(bf16_lo(v.x), bf16_hi(v.x), bf16_lo(v.y), bf16_hi(v.y));
        }
        // quad Q = thread / 4 owns outputs x = 8 (Q & 1) .. + 7 of brick row
        // Q / 2 (y = row mod kBY, z = row / kBY); lane j = thread mod 4 adds
        // input channels 4 j .. 4 j + 3 and finishes outputs 2 j and 2 j + 1
        const int j4 = threadIdx.x & 3, quad = threadIdx.x >> 2;
        const int xh = quad & 1, brow = quad >> 1;
        const int oy = brow % kBY, oz = brow / kBY;
        const float sigma = EPI == E_OUT_U ? 1.0f : (float)(st ? st->sigma : A.sigma[0]);
        // the CTA's bricks b = blockIdx.x, + gridDim.x, ...: brick k is
        // multiplied from buffer k mod 2 while brick k + 1 is staged into the
        // other one, and the epilogue operands of a lane's two nodes are
        // loaded one brick ahead
        const int nb = G.tiles;
        int b = blockIdx.x;
        if (threadIdx.x == 0) {
            mbar_init(&sbar[0], 1);
            mbar_init(&sbar[1], 1);
            mbar_init_fence();
        }
        __syncthreads();
        if (b < nb) stage16_rows_tma(G, brick_of(G, b), A.in, sm, &sbar[0]);
        OutNodes nd = out_nodes<EPI>(A, brick_of(G, b), xh, oy, oz, j4, b < nb);
        for (int k = 0; b < nb; ++k, b += gridDim.x) {
            const unsigned char *cur = sm + (size_t)(k & 1) * kOutStage;
            const int bn = b + gridDim.x;
            if (bn < nb) stage16_rows_tma(G, brick_of(G, bn), A.in, sm + (size_t)((k + 1) & 1) * kOutStage,
                                          &sbar[(k + 1) & 1]);
            // brick b has landed (use k / 2 of its buffer's barrier); brick bn
            // may still be in flight
            if (!mbar_wait_bounded(&sbar[k & 1], (uint32_t)((k >> 1) & 1), A.wait_ns)) {
                // report, then give the copies in flight a second bounded wait
                if (threadIdx.x == 0) {
                    if (st) finish(st, CG_ETIMEOUT);
                    if (A.err) atomicExch(A.err, CG_ETIMEOUT);
                }
                mbar_wait_bounded(&sbar[k & 1], (uint32_t)((k >> 1) & 1), A.wait_ns);
                if (bn < nb) mbar_wait_bounded(&sbar[(k + 1) & 1], (uint32_t)(((k + 1) >> 1) & 1), A.wait_ns);
                return;
            }
            __syncthreads();   // the zero-filled rows (plain stores) too
            // two FP32 partial sums per output (even and odd input channels),
            // one packed f32x2 FMA per channel pair
            uint64_t acc2[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) acc2[i] = 0ull;
            const unsigned char *in0 = cur + (size_t)(xh * 8) * 32 + j4 * 8;
            const ulonglong2 *wt = reinterpret_cast<const ulonglong2 *>(swt) + j4;
#pragma unroll
            for (int g9 = 0; g9 < 9; ++g9) {
                const int dy = g9 % 3 - 1, dz = g9 / 3 - 1;
                // taps (dx, dy, dz), dx = -1, 0, 1: 3 g9, 3 g9 + 1, 3 g9 + 2
                const ulonglong2 wm = wt[4 * (3 * g9)], w0 = wt[4 * (3 * g9 + 1)], wp = wt[4 * (3 * g9 + 2)];
                const unsigned char *in = in0 + ((oy + 1 + dy) + kSY * (oz + 1 + dz)) * kOutRowBytes;
#pragma unroll
                for (int j = 0; j < 10; ++j) {
                    // staged x = 8 xh + j feeds output i = j - 1 - dx
                    const uint2 v = *reinterpret_cast<const uint2 *>(in + j * 32);
                    const uint64_t a01 = bf16x2_f32x2(v.x), a23 = bf16x2_f32x2(v.y);
                    if (j <= 7) acc2[j] = ffma2(wm.y, a23, ffma2(wm.x, a01, acc2[j]));
                    if (j >= 1 && j <= 8) acc2[j - 1] = ffma2(w0.y, a23, ffma2(w0.x, a01, acc2[j - 1]));
                    if (j >= 2) acc2[j - 2] = ffma2(wp.y, a23, ffma2(wp.x, a01, acc2[j - 2]));
                }
            }
            float acc[8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
                acc[i] = __uint_as_float((uint32_t)acc2[i]) + __uint_as_float((uint32_t)(acc2[i] >> 32));
            // the quad's channel partials: a butterfly over its 4 lanes
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], 1);
                acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], 2);
            }
            // z = sigma D^-1/2 u in FP32 (u is the output of BF16 products;
            // FP32 adds nothing to its error), widened for the FP64 dots
            const float u0 = j4 == 0 ? acc[0] : j4 == 1 ? acc[2] : j4 == 2 ? acc[4] : acc[6];
            const float u1 = j4 == 0 ? acc[1] : j4 == 1 ? acc[3] : j4 == 2 ? acc[5] : acc[7];
            if (EPI == E_OUT_U) {
                if (nd.ok0) A.u[nd.i0] = u0;
                if (nd.ok1) A.u[nd.i0 + 1] = u1;
            } else {
                const double z0 = nd.ok0 ? (double)(sigma * nd.d0 * u0) : 0.0;
                const double z1 = nd.ok1 ? (double)(sigma * nd.d1 * u1) : 0.0;
                if (nd.ok0) A.z[nd.i0] = z0;
                if (nd.ok1) A.z[nd.i0 + 1] = z1;
                if (EPI == E_OUT_FCG) {
                    // nodes past the grid have z = r = q = 0: they add 0
                    dzr = fma(z1, nd.r1, fma(z0, nd.r0, dzr));
                    dzq = fma(z1, nd.q1, fma(z0, nd.q0, dzq));
                }
            }
            nd = out_nodes<EPI>(A, brick_of(G, bn), xh, oy, oz, j4, bn < nb);
            __syncthreads();   // buffer k mod 2 is staged again for brick k + 2
        }
    } else {
        const int n = G.n;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
            const double zi = A.dinv[i] * A.r[i];
            A.z[i] = zi;
            dzr = fma(zi, A.r[i], dzr);
            dzq = fma(zi, A.q[i], dzq);
        }
    }
    if (EPI != E_OUT_FCG) return;
    double v[2] = {dzr, dzq}, tot[2];
    __syncthreads();   // the staged input (learned mode) is dead: its space holds the parked sums
    cta_sum2_256(v, reinterpret_cast<double *>(sm), sred);
    if (!last_cta_totals<2>(v, A.partials, &st->counter, tot, &sflag, sred)) return;
    if (threadIdx.x == 0) sswitch = 0;
    if (threadIdx.x == 0) {
        const double zr = tot[0], zq = tot[1];
        st->zr = zr;
        st->zq = zq;
        if (st->mode == kModeLearned && !(zr > 0.0)) {
            // the network gave r.z <= 0 (or not finite): Jacobi-PCG from here on
            st->mode = kModeJacobi;
            st->reverted_at = st->iters;
            st->mode_start = st->iters;
            st->restart = 2;
            st->rho = st->rdr;
            st->beta = 0.0;
            sswitch = 1;
        } else if (!finite_bits(zr)) {
            finish(st, CG_ENAN);
        } else if (!(zr > 0.0)) {
            finish(st, CG_EBREAKDOWN);
        } else {
            st->beta = st->restart ? 0.0 : -st->alpha * zq / st->rho;
            st->rho = zr;
        }
    }
    // on the switch the next SpMV gathers z = D^-1 r (the Jacobi direction),
    // not the network's output: this CTA rewrites z (once per solve at most)
    __syncthreads();
    if (sswitch)
        for (int i = threadIdx.x; i < G.n; i += blockDim.x) A.z[i] = A.dinv[i] * A.r[i];
}

// ------------------------------------------------------- vector kernels
struct VecArgs {
    int n;
    FcgState *st;
    double *x, *r, *z, *p, *q;
    const double *dinv, *dsq;
    const float *dsq32;       // D^-1/2 in FP32 (the network input s = D^-1/2 r)
    const int32_t *pidx;      // padded position of each node
    __nv_bfloat16 *s_in;      // padded network input D^-1/2 r (BF16)
    double *partials;
};

// Warp 0 of the CTA that holds the grid totals {r.r, r.D^-1 r} of the x, r
// update: the iteration count, the residual-norm window of the stall test,
// the stop and stall decisions and the network input's scale sigma.
__device__ __forceinline__ void xr_decide(FcgState *st, const double (&tot)[2], int n) {
    const int lane = threadIdx.x & 31;
    const int k = st->iters + 1;
    const double rn = sqrt(tot[0]);
    const int W = st->window, RS = W + 1;
    if (lane == 0) st->ring[k % RS] = rn;
    __syncwarp();
    double wmin = INFINITY;
    for (int j = lane; j < W && j <= k; j += 32) wmin = fmin(wmin, st->ring[(k - j) % RS]);
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) wmin = fmin(wmin, __shfl_xor_sync(0xffffffffu, wmin, m));
    if (lane != 0) return;
    st->iters = k;
    st->rr = tot[0];
    st->rdr = tot[1];
    if (k >= W) st->best_before = fmin(st->best_before, st->ring[(k - W) % RS]);
    if (!finite_bits(tot[0]) || !finite_bits(tot[1])) {
        finish(st, CG_ENAN);
        return;
    }
    if (rn <= st->tol * st->bnorm) {
        finish(st, CG_OK);
        return;
    }
    if (k >= st->maxit) {
        finish(st, CG_ENOCONV);
        return;
    }
    if (st->mode == kModeLearned && k - st->mode_start >= W && wmin > st->factor * st->best_before) {
        st->mode = kModeJacobi;
        st->reverted_at = k;
        st->mode_start = k;
        st->restart = 1;
    }
    st->sigma = sqrt(tot[1] / (double)n);
    st->sigma_inv = st->sigma > 0.0 ? 1.0 / st->sigma : 0.0;
}

// x += alpha p, r -= alpha q; r.r and r.D^-1 r; stop test, stall test.
// The network input s = D^-1/2 r and r.D^-1 r = s.s are formed in FP32 (s is
// stored in BF16; r.D^-1 r only scales the network input, and after a
// switch to Jacobi-PCG it is the first rho); x, r and r.r stay FP64.
__global__ void __launch_bounds__(kVT) fcg_xr_kernel(VecArgs V) {
    FcgState *st = V.st;
    if (st->done) return;
    __shared__ double sred[2 * 32];
    __shared__ double park[2 * kVT];
    __shared__ int sflag;
    const double alpha = st->alpha;
    double *x = st->x;
    double rr = 0.0;
    float rdr = 0.0f;
    // kXrBatch nodes a thread (stride apart) are loaded before any of them is
    // stored, so their loads are in flight together; the sums still run over
    // the thread's nodes in increasing order
    constexpr int kXrBatch = 4;
    const int stride = gridDim.x * blockDim.x;
    for (int i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < V.n; i0 += kXrBatch * stride) {
        double pv[kXrBatch], xv[kXrBatch], qv[kXrBatch], rv[kXrBatch];
        float dv[kXrBatch];
        int sv[kXrBatch];
#pragma unroll
        for (int j = 0; j < kXrBatch; ++j) {
            const int i = i0 + j * stride;
            if (i < V.n) {
                pv[j] = V.p[i];
                xv[j] = x[i];
                qv[j] = V.q[i];
                rv[j] = V.r[i];
                dv[j] = V.dsq32[i];
                sv[j] = V.pidx[i];
            }
        }
#pragma unroll
        for (int j = 0; j < kXrBatch; ++j) {
            const int i = i0 + j * stride;
            if (i < V.n) {
                x[i] = fma(alpha, pv[j], xv[j]);
                const double ri = fma(-alpha, qv[j], rv[j]);
                V.r[i] = ri;
                const float si = (float)ri * dv[j];
                V.s_in[sv[j]] = __float2bfloat16_rn(si);
                rr = fma(ri, ri, rr);
                rdr = fmaf(si, si, rdr);
            }
        }
    }
    double v[2] = {rr, (double)rdr}, tot[2];
    cta_sum2_256(v, park, sred);
    if (!last_cta_totals<2>(v, V.partials, &st->counter, tot, &sflag, sred)) return;
    if (threadIdx.x < 32) xr_decide(st, tot, V.n);
}

// ---------------------------------------------------------- SpMV kernels
struct EpiSetupL {      // r = b - A x, s_in = D^-1/2 r; r.r, b.b, r.D^-1 r
    const double *b, *dinv, *dsq;
    const int32_t *pidx;
    __nv_bfloat16 *s_in;
    double *r;
    double rr = 0.0, bb = 0.0, rdr = 0.0;
    __device__ __forceinline__ void row(int i, double ax, int) {
        const double bi = b[i], ri = bi - ax;
        r[i] = ri;
        s_in[pidx[i]] = __float2bfloat16_rn((float)(ri * dsq[i]));
        rr = fma(ri, ri, rr);
        bb = fma(bi, bi, bb);
        rdr = fma(ri * dinv[i], ri, rdr);
    }
};
struct EpiQ {           // p = z + beta p, q = A z + beta q (= A p); p.q
    const double *z;    // the gathered vector
    double *p;
    double *q;
    double beta;        // 0 after a restart (p = z)
    double pq = 0.0;
    double zi_ = 0.0, pi_ = 0.0, qi_ = 0.0;   // the row's entries, loaded ahead
    __device__ __forceinline__ void prefetch(int i) {
        zi_ = z[i];
        pi_ = p[i];
        qi_ = q[i];
    }
    __device__ __forceinline__ void row(int i, double az, int) {
        const double qi = fma(beta, qi_, az);
        const double pi = fma(beta, pi_, zi_);
        q[i] = qi;
        p[i] = pi;
        pq = fma(pi, qi, pq);
    }
};
struct EpiTrueL {       // ||b - A x||^2
    const double *b;
    double acc = 0.0;
    __device__ __forceinline__ void row(int i, double ax, int) {
        const double t = b[i] - ax;
        acc = fma(t, t, acc);
    }
};

struct EpiStoreY {      // y = A x
    double *y;
    __device__ __forceinline__ void row(int i, double ax, int) { y[i] = ax; }
};

enum { S_SETUP = 0, S_Q = 1, S_TRUE = 2 };

template <int MODE>
__global__ void __launch_bounds__(kThreads, 1) fcg_spmv_kernel(Params P, FcgState *st, const double *vec,
                                                                double *partials, VecArgs V) {
    if (MODE == S_Q && st->done) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const Smem S = carve_smem(smem_raw);
    __shared__ int sflag;
    init_pipeline(S);
    Pipe pipe;
    double v[3] = {0.0, 0.0, 0.0};
    if (MODE == S_SETUP) {
        EpiSetupL e{st->b, P.dinv, V.dsq, V.pidx, V.s_in, P.r};
        (void)spmv_tiles<0, double, double, double>(P, S, pipe, P.vals, vec, e, true);
        v[0] = e.rr;
        v[1] = e.bb;
        v[2] = e.rdr;
    } else if (MODE == S_Q) {
        EpiQ e{vec, V.p, P.q, st->restart ? 0.0 : st->beta};
        (void)spmv_tiles<0, double, double, double>(P, S, pipe, P.vals, vec, e, true);
        v[0] = e.pq;
    } else {
        EpiTrueL e{st->b};
        (void)spmv_tiles<0, double, double, double>(P, S, pipe, P.vals, vec, e, true);
        v[0] = e.acc;
    }
    drain<double, double>(P, S, pipe, vec);
    block_sum<3>(v, S);
    double tot[3];
    if (!last_cta_totals<3>(v, partials, &st->counter, tot, &sflag, S.red)) return;
    if (threadIdx.x != 0) return;
    if (MODE == S_SETUP) {
        st->rr = tot[0];
        st->bb = tot[1];
        st->rdr = tot[2];
        st->bnorm = sqrt(tot[1]);
        st->iters = 0;
        st->mode = kModeLearned;
        st->restart = 1;
        st->reverted_at = -1;
        st->mode_start = 0;
        st->best_before = INFINITY;
        st->ring[0] = sqrt(tot[0]);
        st->sigma = sqrt(tot[2] / (double)P.n);
        st->sigma_inv = st->sigma > 0.0 ? 1.0 / st->sigma : 0.0;
        st->true_rr = -1.0;
        if (!finite_bits(tot[0]) || !finite_bits(tot[1])) finish(st, CG_ENAN);
        else if (tot[1] == 0.0) finish(st, CG_OK);
        else if (sqrt(tot[0]) <= st->tol * st->bnorm) finish(st, CG_OK);
    } else if (MODE == S_Q) {
        const double pq = tot[0];
        st->pq = pq;
        st->restart = 0;
        if (!finite_bits(pq)) finish(st, CG_ENAN);
        else if (!(pq > 0.0)) finish(st, CG_EBREAKDOWN);
        else st->alpha = st->rho / pq;
    } else {
        st->true_rr = tot[0];
    }
}

// ------------------------------ SpMV step and x, r update in one launch
// The SpMV step and the x, r update of a flexible-CG iteration as one
// cooperative launch (one CTA of 1024 threads per SM) on the SELL-32 copy of
// the matrix.  Warp w of CTA c takes slices cut[c] + w, + 32, ... of the CTA's
// range, and a row is read and written by the same thread in both phases:
//   phase A  q = A z + beta q (= A p), p = z + beta p, partial p.q
//            -> grid barrier; every CTA adds the partials in the same order
//               and forms the same alpha = rho / p.q
//   phase B  x += alpha p, r -= alpha q, the network input D^-1/2 r, partial
//            r.r and r.D^-1 r; the last CTA to finish adds the partials and
//            takes the stop and stall decisions
// The arithmetic of fcg_spmv_kernel<S_Q> followed by fcg_xr_kernel, with one
// launch and one pass over p, q fewer; the SELL-32 SpMV streams each row's
// entries in coalesced batches with no staging.
struct FcgSellArgs {
    Params P;             // partials (set 0: p.q; set 1: r.r, r.D^-1 r), wait bound, error block
    SellMatrix M;
    const int32_t *cut;   // CTA c owns slices cut[c] .. cut[c + 1] - 1
    VecArgs V;
};

__device__ __forceinline__ unsigned int atom_add_acq_rel(unsigned int *a, unsigned int v) {
    unsigned int old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(a), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ void st_relaxed(unsigned int *a, unsigned int v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release(unsigned int *a, unsigned int v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}

// A grid barrier that resets itself, for a kernel launched many times in one
// graph.  Thread 0 of each CTA reads the generation word, then arrives on the
// counter (acquire-release); the last to arrive clears the counter and
// publishes the next generation (release); the others wait for it (acquire,
// bounded by wait_ns).  The __syncthreads after the call carries the
// ordering to the rest of the CTA.  Returns 1 when the barrier has passed.
// phantom (a test knob, 0 in use) counts CTAs that never arrive, so that the
// waits run out.
__device__ __forceinline__ int fcg_grid_sync(FcgState *st, unsigned long long wait_ns, int phantom) {
    const unsigned int gen = ld_acquire(&st->bar_gen);
    if (atom_add_acq_rel(&st->bar_count, 1u) == gridDim.x - 1 + (unsigned)phantom) {
        st_relaxed(&st->bar_count, 0u);
        st_release(&st->bar_gen, gen + 1u);
        return 1;
    }
    if (ld_acquire(&st->bar_gen) != gen) return 1;
    const unsigned long long t0 = global_ns();
    unsigned int spins = 0;
    while (ld_acquire(&st->bar_gen) == gen) {
        if ((++spins & 63u) == 0 && global_ns() - t0 > wait_ns) return 0;
    }
    return 1;
}

__global__ void __launch_bounds__(kSellSolveThreads, 1) fcg_sell_kernel(FcgSellArgs F) {
    const VecArgs &V = F.V;
    FcgState *st = V.st;
    if (st->done) return;   // written only by earlier kernels: the same in every CTA
    __shared__ double red[2 * kSellSolveThreads];
    __shared__ double quarter[8];
    __shared__ double bcast[1];
    __shared__ int ctl[3];
    constexpr int kW = kSellSolveThreads / 32;
    const int tid = threadIdx.x, lane = tid & 31;
    const int t0 = F.cut[blockIdx.x] + (tid >> 5), t1 = F.cut[blockIdx.x + 1];
    const int n = V.n;
    // read before the barrier; CTA 0 changes restart only after it
    const double beta = st->restart ? 0.0 : st->beta;
    const double rho = st->rho;
    double *const x = st->x;

    // phase A: q = A z + beta q (= A p), p = z + beta p; p . q
    double v1[1] = {0.0};
    for (int t = t0; t < t1; t += kW) {
        const double az = sell_slice_sum<kSellUnrollMem>(F.M, t, V.z, 0.0);
        const int row = t * 32 + lane;
        if (row < n) {
            const double qi = fma(beta, V.q[row], az);
            const double pi = fma(beta, V.p[row], V.z[row]);
            V.q[row] = qi;
            V.p[row] = pi;
            v1[0] = fma(pi, qi, v1[0]);
        }
    }
    block_sum_1k<1>(v1, red, quarter);
    publish_partials<1>(F.P, 0, v1);
    if (tid == 0) {
        const int ok = fcg_grid_sync(st, F.P.wait_ns, F.P.phantom);
        if (!ok) {
            set_error(F.P.st, CG_ETIMEOUT, 3);
            finish(st, CG_ETIMEOUT);
        }
        ctl[0] = ok;
    }
    __syncthreads();
    if (!ctl[0]) return;
    double sg[1];
    grid_totals_1k<1>(F.P, 0, sg, quarter);
    if (tid == 0) {
        const double pq = sg[0];
        const int go = finite_bits(pq) && pq > 0.0;
        const double alpha = go ? rho / pq : 0.0;
        if (blockIdx.x == 0) {
            st->pq = pq;
            st->restart = 0;
            if (!finite_bits(pq)) finish(st, CG_ENAN);
            else if (!(pq > 0.0)) finish(st, CG_EBREAKDOWN);
            else st->alpha = alpha;
        }
        bcast[0] = alpha;
        ctl[1] = go;
    }
    __syncthreads();
    if (!ctl[1]) return;
    const double alpha = bcast[0];

    // phase B: x += alpha p, r -= alpha q, s = D^-1/2 r (FP32, stored in
    // BF16 at its padded position); r.r in FP64, r.D^-1 r = s.s in FP32
    double rr = 0.0;
    float rdr = 0.0f;
    for (int t = t0; t < t1; t += kW) {
        const int row = t * 32 + lane;
        if (row < n) {
            const double ri = fma(-alpha, V.q[row], V.r[row]);
            x[row] = fma(alpha, V.p[row], x[row]);
            V.r[row] = ri;
            const float si = (float)ri * V.dsq32[row];
            V.s_in[V.pidx[row]] = __float2bfloat16_rn(si);
            rr = fma(ri, ri, rr);
            rdr = fmaf(si, si, rdr);
        }
    }
    double v2[2] = {rr, (double)rdr};
    block_sum_1k<2>(v2, red, quarter);
    publish_partials<2>(F.P, 1, v2);
    if (tid == 0) {
        __threadfence();
        ctl[2] = atomicAdd(&st->counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!ctl[2]) return;
    __threadfence();
    if (tid < 32) {
        double tot[2];
        grid_totals<2>(F.P, 1, tot);
        if (tid == 0) st->counter = 0u;
        xr_decide(st, tot, n);
    }
}

// Plain y = A x for training (no reductions).
__global__ void __launch_bounds__(kSellThreads) spmv_store_kernel(SellMatrix M, const double *x, double *y) {
    EpiStoreY e{y};
    sell_rows(M, x, e);
}

// ------------------------------------------------------------ training
struct TrainArgs {
    Geo G;
    const float *r, *e;       // the pair (node order)
    const double *dinv, *dsq;
    double *scal;             // [0] sigma, [1] 1/sigma, [2] loss sum of the step, [3] counter space
    unsigned int *counter;
    double *partials;
    __nv_bfloat16 *shat;      // padded, 1 channel
    float *ehat;              // node order
    const float *u;           // network output (node order)
    float *v;                 // u - e_hat
    double *t;                // D^-1/2 v (SpMV input)
    const double *y;          // A t
    __nv_bfloat16 *du;        // padded, 1 channel: A_hat v (n times the loss gradient)
    const int32_t *pidx;      // padded position of each node
};

// sigma = rms(D^-1/2 v) over a node-order vector (FP32 pair or FP64 residual).
template <class VT>
__global__ void __launch_bounds__(kVT) sigma_kernel(int n, const VT *v, const double *dinv, double *scal,
                                                    unsigned int *counter, double *partials) {
    __shared__ double sred[32];
    __shared__ int sflag;
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double vi = (double)v[i];
        acc = fma(vi * dinv[i], vi, acc);
    }
    double a[1] = {acc}, tot[1];
    cta_sum<1>(a, sred);
    if (!last_cta_totals<1>(a, partials, counter, tot, &sflag, sred)) return;
    if (threadIdx.x == 0) {
        const double sigma = sqrt(tot[0] / (double)n);
        scal[0] = sigma;
        scal[1] = sigma > 0.0 ? 1.0 / sigma : 0.0;
    }
}

// s_hat (padded BF16) and e_hat = D^1/2 e / sigma (FP32, node order).
__global__ void __launch_bounds__(kVT) pair_input_kernel(TrainArgs T) {
    const double sinv = T.scal[1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < T.G.n; i += gridDim.x * blockDim.x) {
        T.shat[T.pidx[i]] = __float2bfloat16_rn((float)((double)T.r[i] * T.dsq[i] * sinv));
        T.ehat[i] = (float)((double)T.e[i] / T.dsq[i] * sinv);
    }
}

// v = u - e_hat, t = D^-1/2 v.
__global__ void __launch_bounds__(kVT) loss_prep_kernel(TrainArgs T) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < T.G.n; i += gridDim.x * blockDim.x) {
        const float vi = T.u[i] - T.ehat[i];
        T.v[i] = vi;
        T.t[i] = T.dsq[i] * (double)vi;
    }
}

// w = D^-1/2 A t = A_hat v; loss += v.w / 2n; du = w (padded BF16).
__global__ void __launch_bounds__(kVT) loss_kernel(TrainArgs T) {
    __shared__ double sred[32];
    __shared__ int sflag;
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < T.G.n; i += gridDim.x * blockDim.x) {
        const double wi = T.dsq[i] * T.y[i];
        acc = fma((double)T.v[i], wi, acc);
        T.du[T.pidx[i]] = __float2bfloat16_rn((float)wi);
    }
    double a[1] = {acc}, tot[1];
    cta_sum<1>(a, sred);
    if (!last_cta_totals<1>(a, T.partials, T.counter, tot, &sflag, sred)) return;
    if (threadIdx.x == 0) T.scal[2] += 0.5 * tot[0] / (double)T.G.n;
}

// dag = dg * g (1 - g) over the whole padded 16-channel field (zero halos stay zero).
__global__ void __launch_bounds__(kVT) gate_grad_kernel(long long count, const float *dg, const __nv_bfloat16 *gate,
                                                       __nv_bfloat16 *dag) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < count;
         k += (long long)gridDim.x * blockDim.x) {
        const float gv = __bfloat162float(gate[k]);
        dag[k] = __float2bfloat16_rn(dg[k] * gv * (1.0f - gv));
    }
}

struct WgArgs {
    Geo G;
    const __nv_bfloat16 *dy;   // padded 16-channel field
    const __nv_bfloat16 *x;    // padded field (16 channels for wgrad16, 1 for wgrad1)
    float *part;               // gridDim.x x CG_LEARN_PARAMS partial gradients
    int off;                   // parameter offset of this weight ([o][c][t] or [o][t])
    int bias_off;              // wgrad1: offset of the channel sums of dy (-1: none)
    int add;                   // 0: part = ..., 1: part += ...
};

// Stages the gradient brick dy (16 x 8 x 4 positions, no halo): row
// (yl, zl) at kBX (zl * kBY + yl), swizzled like the input.
__device__ __forceinline__ void stage_dy(const Geo &G, const Brick &B, const __nv_bfloat16 *dy, unsigned char *sdy) {
    constexpr int kChunks = kBX * 2;
    for (int c = threadIdx.x; c < kRows * kChunks; c += blockDim.x) {
        const int row = c / kChunks, k = c - row * kChunks;
        const int xr = k >> 1, h = k & 1;
        const int yl = row % kBY, zl = row / kBY;
        const int R = row * kBX + xr;
        unsigned char *dst = sdy + R * 32 + ((h ^ ((R >> 2) & 1)) << 4);
        long long pos0;
        // positions past the grid in x would read the next row: they are zeroed
        if (staged_row(G, B, yl + 1, zl + 1, pos0) && B.x0 + xr < G.nx)
            cp_async16(dst, dy + (pos0 + 1 + xr) * kCh + h * 8);
        else
            *reinterpret_cast<uint4 *>(dst) = make_uint4(0u, 0u, 0u, 0u);
    }
}

// Staged input row of dy row `row` (= zl * kBY + yl), shifted by a tap.
__device__ __forceinline__ int x_row(int row, int dx, int dy, int dz) {
    const int yl = row % kBY, zl = row / kBY;
    return ((zl + 1 + dz) * kSY + (yl + 1 + dy)) * kSX + 1 + dx;
}

// G[o][c][t] = sum_p dy[o, p] x[c, p + off(t)] for 16-channel dy and x: a
// GEMM over positions (M = o, N = c, K = p) per tap; warp w owns taps
// w, w + 8, ...  Persistent over bricks; the CTA's sums go to part[blockIdx.x].
// dy is zero off the interior nodes, so dropped positions add nothing.
__global__ void __launch_bounds__(kCT) wgrad16_kernel(WgArgs W) {
    extern __shared__ __align__(128) unsigned char sm[];
    const Geo &G = W.G;
    unsigned char *sdy = sm + kStage16;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, g = lane >> 2, t4 = lane & 3;
    constexpr int kWarpsC = kCT / 32;
    constexpr int kMaxT = (kTaps + kWarpsC - 1) / kWarpsC;
    float acc[kMaxT][2][4];
#pragma unroll
    for (int i = 0; i < kMaxT; ++i)
#pragma unroll
        for (int nb = 0; nb < 2; ++nb)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[i][nb][k] = 0.0f;
    const uint32_t in_base = smem_u32(sm), dy_base = smem_u32(sdy);
    const int a_pos = (lane & 7) + ((lane >> 4) << 3), a_half = (lane >> 3) & 1;
    const int b_pos = (lane & 7) + (((lane >> 3) & 1) << 3), b_half = lane >> 4;
    for (int tile = blockIdx.x; tile < G.tiles; tile += gridDim.x) {
        const Brick B = brick_of(G, tile);
        stage16(G, B, W.x, sm);
        stage_dy(G, B, W.dy, sdy);
        cp_async_wait_all();
        __syncthreads();
        for (int row = 0; row < kRows; ++row) {
            uint32_t a[4];
            ldsm_x4_t(a, row_addr(dy_base, row * kBX + a_pos, a_half));
#pragma unroll
            for (int i = 0; i < kMaxT; ++i) {
                const int t = w + kWarpsC * i;
                if (t < kTaps) {
                    uint32_t b[4];
                    ldsm_x4_t(b, row_addr(in_base, x_row(row, tap_dx(t), tap_dy(t), tap_dz(t)) + b_pos, b_half));
                    mma_bf16(acc[i][0], a, b[0], b[1]);
                    mma_bf16(acc[i][1], a, b[2], b[3]);
                }
            }
        }
        __syncthreads();
    }
    float *part = W.part + (size_t)blockIdx.x * CG_LEARN_PARAMS + W.off;
#pragma unroll
    for (int i = 0; i < kMaxT; ++i) {
        const int t = w + kWarpsC * i;
        if (t >= kTaps) continue;
#pragma unroll
        for (int nb = 0; nb < 2; ++nb)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int o = g + 8 * (k >> 1), c = nb * 8 + 2 * t4 + (k & 1);
                float *dst = part + (o * kCh + c) * kTaps + t;
                *dst = W.add ? *dst + acc[i][nb][k] : acc[i][nb][k];
            }
    }
}

// G[o][t] = sum_p dy[o, p] x[p + off(t)] for 16-channel dy and a 1-channel
// x (taps are the GEMM's N dimension, 4 blocks of 8; "tap" 27 multiplies
// by one and gives the channel sums of dy when bias_off >= 0).  Warps split
// the rows of a brick and add their sums in shared memory at the end.
__global__ void __launch_bounds__(kCT) wgrad1_kernel(WgArgs W) {
    extern __shared__ __align__(128) unsigned char sm[];
    const Geo &G = W.G;
    constexpr int kWarpsC = kCT / 32;
    uint16_t *xs = reinterpret_cast<uint16_t *>(sm);
    unsigned char *sdy = sm + kStage1;
    float *sacc = reinterpret_cast<float *>(sdy + kDyTile);   // [warps][16][32]
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, g = lane >> 2, t4 = lane & 3;
    float acc[4][4];
#pragma unroll
    for (int nb = 0; nb < 4; ++nb)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[nb][k] = 0.0f;
    const uint32_t dy_base = smem_u32(sdy);
    const int a_pos = (lane & 7) + ((lane >> 4) << 3), a_half = (lane >> 3) & 1;
    int tkind[4];   // 0 tap, 1 constant one, 2 zero
    int tt_of[4];
#pragma unroll
    for (int nb = 0; nb < 4; ++nb) {
        const int t = nb * 8 + g;
        tkind[nb] = t < kTaps ? 0 : (t == kTaps && W.bias_off >= 0 ? 1 : 2);
        tt_of[nb] = t < kTaps ? t : kCentre;
    }
    for (int tile = blockIdx.x; tile < G.tiles; tile += gridDim.x) {
        const Brick B = brick_of(G, tile);
        stage1(G, B, W.x, xs);
        stage_dy(G, B, W.dy, sdy);
        cp_async_wait_all();
        __syncthreads();
        for (int row = w; row < kRows; row += kWarpsC) {
            uint32_t a[4];
            ldsm_x4_t(a, row_addr(dy_base, row * kBX + a_pos, a_half));
#pragma unroll
            for (int nb = 0; nb < 4; ++nb) {
                uint32_t b0, b1;
                if (tkind[nb] == 0) {
                    const int tt = tt_of[nb];
                    const uint16_t *xp = xs + x_row(row, tap_dx(tt), tap_dy(tt), tap_dz(tt)) + 2 * t4;
                    b0 = pack_raw(xp[0], xp[1]);
                    b1 = pack_raw(xp[8], xp[9]);
                } else if (tkind[nb] == 1) {
                    b0 = b1 = 0x3F803F80u;   // BF16 ones
                } else {
                    b0 = b1 = 0u;
                }
                mma_bf16(acc[nb], a, b0, b1);
            }
        }
        __syncthreads();
    }
    // sum the warps' accumulators: sacc[w][o][tap]
#pragma unroll
    for (int nb = 0; nb < 4; ++nb)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int o = g + 8 * (k >> 1), tap = nb * 8 + 2 * t4 + (k & 1);
            sacc[(w * 16 + o) * 32 + tap] = acc[nb][k];
        }
    __syncthreads();
    float *part = W.part + (size_t)blockIdx.x * CG_LEARN_PARAMS;
    for (int idx = threadIdx.x; idx < 16 * 32; idx += blockDim.x) {
        const int o = idx >> 5, tap = idx & 31;
        float s = 0.0f;
#pragma unroll
        for (int ww = 0; ww < kWarpsC; ++ww) s += sacc[(ww * 16 + o) * 32 + tap];
        float *dst = nullptr;
        if (tap < kTaps) dst = part + W.off + o * kTaps + tap;
        else if (tap == kTaps && W.bias_off >= 0) dst = part + W.bias_off + o;
        if (dst) *dst = W.add ? *dst + s : s;
    }
}

// grad[j] += sum over CTAs (in order) of part[cta][j].
__global__ void __launch_bounds__(kVT) grad_reduce_kernel(const float *part, int nparts, float *grad) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= CG_LEARN_PARAMS) return;
    float s = 0.0f;
    for (int c = 0; c < nparts; ++c) s += part[(size_t)c * CG_LEARN_PARAMS + j];
    grad[j] += s;
}

struct NetDev {
    float *theta, *m, *v, *grad;
    __nv_bfloat16 *k1in, *k1t, *k2, *k2t, *kgin;
    float *bg;
    double *loss_hist;
};

// Packs parameter j into the kernels' BF16 layouts.
__device__ __forceinline__ void pack_param(const NetDev &N, int j, float th) {
    const __nv_bfloat16 b = __float2bfloat16_rn(th);
    if (j < kOffW2) {
        const int o = j / kTaps, t = j % kTaps;
        N.k1in[o * kTapsPad + t] = b;
        N.k1t[(kTaps - 1 - t) * kCh + o] = b;
    } else if (j < kOffWg) {
        const int jj = j - kOffW2;
        const int o = jj / (kCh * kTaps), c = (jj / kTaps) % kCh, t = jj % kTaps;
        N.k2[(t * kCh + o) * kCh + c] = b;
        N.k2t[((kTaps - 1 - t) * kCh + c) * kCh + o] = b;
    } else if (j < kOffBg) {
        const int jj = j - kOffWg;
        N.kgin[(jj / kTaps) * kTapsPad + jj % kTaps] = b;
    } else {
        N.bg[j - kOffBg] = th;
    }
}

// Adam step (lr > 0) on grad * scale, or (lr == 0) only the packing; clears
// grad; records the step's mean loss.
__global__ void __launch_bounds__(kVT) adam_kernel(NetDev N, float scale, float lr, float bc1, float bc2,
                                                   double *scal, double loss_scale, int step_slot) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j == 0 && step_slot >= 0) {
        N.loss_hist[step_slot] = scal[2] * loss_scale;
        scal[2] = 0.0;
    }
    if (j >= CG_LEARN_PARAMS) return;
    float th = N.theta[j];
    if (lr > 0.0f) {
        const float gr = N.grad[j] * scale;
        const float m = 0.9f * N.m[j] + 0.1f * gr;
        const float v = 0.999f * N.v[j] + 0.001f * gr * gr;
        N.m[j] = m;
        N.v[j] = v;
        th -= lr * (m / bc1) / (sqrtf(v / bc2) + 1e-8f);
        N.theta[j] = th;
    }
    N.grad[j] = 0.0f;
    pack_param(N, j, th);
}

// r_s = b - A x, e_s = xstar - x (as floats).
__global__ void __launch_bounds__(kVT) pair_record_kernel(int n, const double *b, const double *xstar,
                                                          const double *x, const double *ax, float *r, float *e) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        r[i] = (float)(b[i] - ax[i]);
        e[i] = (float)(xstar[i] - x[i]);
    }
}

// s_in = D^-1/2 r at the padded positions (the network input before 1/sigma).
__global__ void __launch_bounds__(kVT) scatter_s_kernel(int n, const double *r, const double *dsq,
                                                        const int32_t *pidx, __nv_bfloat16 *s_in) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        s_in[pidx[i]] = __float2bfloat16_rn((float)(r[i] * dsq[i]));
}

__global__ void __launch_bounds__(kVT) dsq_kernel(int n, const double *dinv, double *dsq, float *dsq32) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        dsq[i] = sqrt(dinv[i]);
        dsq32[i] = (float)dsq[i];
    }
}

}  // namespace

// ================================================================= host

struct cg_net {
    int device = 0;
    cudaStream_t stream = nullptr;
    NetDev d{};
    void *block = nullptr;
    long long step = 0;
    // training workspace (allocated on first use, for one grid)
    Geo tg{};
    bool have_train = false;
    std::vector<void *> tallocs;
    __nv_bfloat16 *shat = nullptr, *a1 = nullptr, *h1 = nullptr, *h2 = nullptr, *kpre = nullptr, *k1 = nullptr;
    __nv_bfloat16 *du = nullptr, *dk = nullptr, *dh2 = nullptr, *da1 = nullptr, *dag = nullptr;
    float *dg = nullptr, *u = nullptr, *ehat = nullptr, *v = nullptr, *part = nullptr;
    double *t = nullptr, *y = nullptr, *scal = nullptr, *partials = nullptr;
    unsigned int *counter = nullptr;
    int loss_cap_n = 0;
    int wg_ctas = 0;
    int vgrid = 0;
};

namespace gbcg {

struct LearnCtx {
    cg_net *net = nullptr;
    Geo G{};
    int window = 50;
    double factor = 0.9;
    std::vector<void *> allocs;
    __nv_bfloat16 *lognu_in = nullptr, *gates = nullptr, *h1 = nullptr, *h2 = nullptr, *k1 = nullptr;
    __nv_bfloat16 *s_in = nullptr;   // padded D^-1/2 r (network input)
    int32_t *pidx = nullptr;         // padded position of each node
    double *dsq = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
    float *dsq32 = nullptr;          // D^-1/2 in FP32
    double *partials = nullptr, *sigma = nullptr;
    unsigned int *counter = nullptr;
    int *conv_err = nullptr;         // timeout report of the tensor-core convolution (apply)
    FcgState *st = nullptr;
    DevStatus *dst = nullptr;
    FcgState *st_host = nullptr;     // pinned
    FcgFlags *flags_host = nullptr;  // pinned, 2 slots
    DevStatus *dst_host = nullptr;   // pinned, 2 slots
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    cg_net *graph_net = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    int vgrid = 0;
    int fused = 0;                   // 1: the SpMV step and the x, r update run as fcg_sell_kernel
};

}  // namespace gbcg

namespace {

int sm_count(int dev) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

// CTAs of a 16 -> 1 convolution launch: persistent, as many as are resident
// at once (each loops over its share of the bricks), at most one per brick.
template <int EPI>
int convout_grid(const Geo &G) {
    int dev = 0, occ = 0;
    cudaGetDevice(&dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, convout_kernel<EPI>, kCT, convout_smem(G)) != cudaSuccess ||
        occ < 1)
        occ = 1;
    return std::max(1, std::min(G.tiles, occ * sm_count(dev)));
}

template <class T>
int ctx_alloc(std::vector<void *> &allocs, T **p, size_t count, bool zero = true) {
    *p = nullptr;
    void *v = nullptr;
    cudaError_t e = cudaMalloc(&v, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(e);
    allocs.push_back(v);
    if (zero && cudaMemset(v, 0, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) return CG_ECUDA;
    *p = static_cast<T *>(v);
    return CG_OK;
}

size_t act_count(const Geo &G, int ch) { return (size_t)(G.npad + kSlack) * ch; }

// Lets every kernel use all the shared memory a block may opt in to, minus
// its static shared memory (the two count against the same limit).
int set_smem_limits() {
    static int done = 0;
    if (done) return CG_OK;
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return CG_ECUDA;
    cudaError_t e = cudaSuccess;
    auto set = [&](const void *f) {
        cudaFuncAttributes fa{};
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, f);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     optin - (int)fa.sharedSizeBytes);
    };
    // the SELL SpMVs stage nothing: all of the SM's storage goes to L1, where
    // the gathers of x find the neighbours other warps already loaded
    auto l1 = [&](const void *f) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxL1);
    };
    set((const void *)conv16_kernel<E_STORE>);
    set((const void *)conv16_kernel<E_GATE>);
    set((const void *)conv16_kernel<E_GATE_PRE>);
    set((const void *)conv16_kernel<E_BWD_GATE>);
    set((const void *)conv16tc_kernel<E_STORE>);
    set((const void *)conv16tc_kernel<E_GATE>);
    set((const void *)convout_kernel<E_OUT_U>);
    set((const void *)convout_kernel<E_OUT_Z>);
    set((const void *)convout_kernel<E_OUT_FCG>);
    set((const void *)wgrad16_kernel);
    set((const void *)wgrad1_kernel);
    set((const void *)fcg_spmv_kernel<S_SETUP>);
    set((const void *)fcg_spmv_kernel<S_Q>);
    set((const void *)fcg_spmv_kernel<S_TRUE>);
    l1((const void *)spmv_store_kernel);
    set((const void *)conv1_kernel<E_GATE>);
    set((const void *)conv1_kernel<E_SIGMOID>);
    set((const void *)conv1_kernel<E_GATE_PRE>);
    set((const void *)conv1_kernel<E_BWD_GATE>);

    if (e != cudaSuccess) return CG_ECUDA;
    done = 1;
    return CG_OK;
}

ConvArgs conv_args(const Geo &G) {
    ConvArgs A{};
    A.G = G;
    A.wait_ns = 5000000000ull;
    return A;
}

// Gates g = sigmoid(Cg(lognu / 8) + bg) of an instance with the net's current parameters.
void launch_gates(const LearnCtx *L, const cg_net *net, cudaStream_t s) {
    ConvArgs A = conv_args(L->G);
    A.in = L->lognu_in;
    A.w = net->d.kgin;
    A.bias = net->d.bg;
    A.out = L->gates;
    conv1_kernel<E_SIGMOID><<<L->G.tiles, kCT, conv1_smem(L->G), s>>>(A);
}

Params learn_params(cg_handle *h, LearnCtx *L) {
    Params P = base_params(h);
    P.r = L->r;
    P.q = L->q;
    P.z = L->z;
    P.st = L->dst;
    return P;
}

VecArgs vec_args(cg_handle *h, LearnCtx *L) {
    VecArgs V{};
    V.n = L->G.n;
    V.st = L->st;
    V.r = L->r;
    V.z = L->z;
    V.p = L->p;
    V.q = L->q;
    V.dinv = h->dinv;
    V.dsq = L->dsq;
    V.dsq32 = L->dsq32;
    V.pidx = L->pidx;
    V.s_in = L->s_in;
    V.partials = L->partials;
    return V;
}

// One flexible-CG iteration: five launches (six without the fused kernel).
void enqueue_body(cg_handle *h, LearnCtx *L, cudaStream_t s) {
    const Geo &G = L->G;
    const cg_net *net = L->net;
    ConvArgs A = conv_args(G);
    A.st = L->st;
    A.dsq = L->dsq;
    A.dsq32 = L->dsq32;
    A.gate = L->gates;
    // h1 = g * C1(D^-1/2 r) / sigma
    A.in = L->s_in;
    A.w = net->d.k1in;
    A.out = L->h1;
    conv1_kernel<E_GATE><<<G.tiles, kCT, conv1_smem(G), s>>>(A);
    // h2 = C2(h1)
    A.in = L->h1;
    A.w = net->d.k2;
    A.out = L->h2;
    A.wait_ns = (unsigned long long)(h->opts.wait_limit_s * 1e9);
    conv16tc_kernel<E_STORE><<<G.ttiles, kCT, conv16tc_smem(G), s>>>(A);
    // k1 = g * C2^T(h2)
    A.in = L->h2;
    A.w = net->d.k2t;
    A.out = L->k1;
    conv16tc_kernel<E_GATE><<<G.ttiles, kCT, conv16tc_smem(G), s>>>(A);
    // z = sigma D^-1/2 C1^T(k1) (or D^-1 r), z.r, z.q, beta
    A.in = L->k1;
    A.w = net->d.k1t;
    A.z = L->z;
    A.r = L->r;
    A.q = L->q;
    A.dinv = h->dinv;
    A.partials = L->partials;
    convout_kernel<E_OUT_FCG><<<convout_grid<E_OUT_FCG>(G), kCT, convout_smem(G), s>>>(A);
    const VecArgs V = vec_args(h, L);
    if (L->fused) {
        // SpMV step and x, r update in one cooperative launch (SELL-32)
        FcgSellArgs F{learn_params(h, L), sell_of(h), h->sell_cut, V};
        void *args[] = {&F};
        cudaLaunchCooperativeKernel((const void *)fcg_sell_kernel, dim3(h->ctas), dim3(kSellSolveThreads), args, 0,
                                    s);
    } else {
        // p = z + beta p and q = A z + beta q in the SpMV's epilogue (it gathers z)
        fcg_spmv_kernel<S_Q><<<h->ctas, kThreads, kSmemBytes, s>>>(learn_params(h, L), L->st, L->z, L->partials, V);
        fcg_xr_kernel<<<L->vgrid, kVT, 0, s>>>(V);
    }
}

// Kernels of one flexible-CG iteration (one graph body).
int body_kernels(const LearnCtx *L) { return L->fused ? 5 : 6; }

int capture(cg_handle *h, LearnCtx *L) {
    if (L->graph) {
        cudaGraphExecDestroy(L->graph);
        L->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(L->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return CG_ECUDA;
    for (int u = 0; u < kUnroll; ++u) enqueue_body(h, L, L->cap_stream);
    cudaError_t e = cudaStreamEndCapture(L->cap_stream, &g);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&L->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        L->graph = nullptr;
        cudaGetLastError();
        return CG_ECUDA;
    }
    L->graph_net = L->net;
    return CG_OK;
}

void free_ctx(LearnCtx *L) {
    if (!L) return;
    if (L->graph) cudaGraphExecDestroy(L->graph);
    if (L->cap_stream) cudaStreamDestroy(L->cap_stream);
    for (cudaEvent_t e : {L->ev[0], L->ev[1], L->t0, L->t1})
        if (e) cudaEventDestroy(e);
    for (void *p : L->allocs) cudaFree(p);
    if (L->st_host) cudaFreeHost(L->st_host);
    if (L->flags_host) cudaFreeHost(L->flags_host);
    if (L->dst_host) cudaFreeHost(L->dst_host);
    delete L;
}

bool finite_params(const float *p) {
    for (int j = 0; j < CG_LEARN_PARAMS; ++j)
        if (!std::isfinite(p[j])) return false;
    return true;
}

int upload_params(cg_net *net, const float *params) {
    if (cudaMemcpyAsync(net->d.theta, params, sizeof(float) * CG_LEARN_PARAMS, cudaMemcpyHostToDevice,
                        net->stream) != cudaSuccess ||
        cudaMemsetAsync(net->d.m, 0, sizeof(float) * CG_LEARN_PARAMS, net->stream) != cudaSuccess ||
        cudaMemsetAsync(net->d.v, 0, sizeof(float) * CG_LEARN_PARAMS, net->stream) != cudaSuccess)
        return CG_ECUDA;
    net->step = 0;
    adam_kernel<<<(CG_LEARN_PARAMS + kVT - 1) / kVT, kVT, 0, net->stream>>>(net->d, 0.0f, 0.0f, 1.0f, 1.0f, nullptr,
                                                                             0.0, -1);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(net->stream) != cudaSuccess) return CG_ECUDA;
    return CG_OK;
}

// Training workspace of the net for one grid.
int ensure_train(cg_net *net, const Geo &G, int ninst_ctas) {
    if (net->have_train && net->tg.nx == G.nx && net->tg.ny == G.ny && net->tg.nz == G.nz) return CG_OK;
    for (void *p : net->tallocs) cudaFree(p);
    net->tallocs.clear();
    net->have_train = false;
    net->tg = G;
    net->wg_ctas = std::min(G.tiles, 2 * sm_count(net->device));
    net->vgrid = std::min((G.n + kVT - 1) / kVT, 4 * sm_count(net->device));
    const size_t a16 = act_count(G, kCh), a1 = act_count(G, 1);
    auto &A = net->tallocs;
    int rc;
    if ((rc = ctx_alloc(A, &net->shat, a1)) || (rc = ctx_alloc(A, &net->a1, a16)) || (rc = ctx_alloc(A, &net->h1, a16)) ||
        (rc = ctx_alloc(A, &net->h2, a16)) || (rc = ctx_alloc(A, &net->kpre, a16)) ||
        (rc = ctx_alloc(A, &net->k1, a16)) || (rc = ctx_alloc(A, &net->du, a1)) || (rc = ctx_alloc(A, &net->dk, a16)) ||
        (rc = ctx_alloc(A, &net->dh2, a16)) || (rc = ctx_alloc(A, &net->da1, a16)) ||
        (rc = ctx_alloc(A, &net->dag, a16)) || (rc = ctx_alloc(A, &net->dg, a16)) ||
        (rc = ctx_alloc(A, &net->u, (size_t)G.n)) || (rc = ctx_alloc(A, &net->ehat, (size_t)G.n)) ||
        (rc = ctx_alloc(A, &net->v, (size_t)G.n)) || (rc = ctx_alloc(A, &net->t, (size_t)G.n + 16)) ||
        (rc = ctx_alloc(A, &net->y, (size_t)G.n)) || (rc = ctx_alloc(A, &net->scal, 8)) ||
        (rc = ctx_alloc(A, &net->counter, 4)) ||
        (rc = ctx_alloc(A, &net->partials, (size_t)4 * std::max({net->vgrid, ninst_ctas, 1}))) ||
        (rc = ctx_alloc(A, &net->part, (size_t)net->wg_ctas * CG_LEARN_PARAMS)))
        return rc;
    net->have_train = true;
    return CG_OK;
}

// Loss and gradient of one pair, added to net->d.grad and scal[2] (stream net->stream).
void enqueue_sample(cg_net *net, cg_handle *h, const float *r, const float *e) {
    LearnCtx *L = h->learn;
    const Geo &G = L->G;
    cudaStream_t s = net->stream;
    TrainArgs T{};
    T.G = G;
    T.r = r;
    T.e = e;
    T.dinv = h->dinv;
    T.dsq = L->dsq;
    T.scal = net->scal;
    T.counter = net->counter;
    T.partials = net->partials;
    T.shat = net->shat;
    T.ehat = net->ehat;
    T.u = net->u;
    T.v = net->v;
    T.t = net->t;
    T.y = net->y;
    T.du = net->du;
    T.pidx = L->pidx;
    const int vg = net->vgrid;
    sigma_kernel<float><<<vg, kVT, 0, s>>>(G.n, r, h->dinv, net->scal, net->counter, net->partials);
    pair_input_kernel<<<vg, kVT, 0, s>>>(T);
    launch_gates(L, net, s);
    ConvArgs A = conv_args(G);
    A.gate = L->gates;
    // forward, keeping the pre-gate fields
    A.in = net->shat;
    A.w = net->d.k1in;
    A.out = net->h1;
    A.pre = net->a1;
    conv1_kernel<E_GATE_PRE><<<G.tiles, kCT, conv1_smem(G), s>>>(A);
    A.in = net->h1;
    A.w = net->d.k2;
    A.out = net->h2;
    conv16_kernel<E_STORE><<<G.tiles, kCT, conv16_smem(G), s>>>(A);
    A.in = net->h2;
    A.w = net->d.k2t;
    A.out = net->k1;
    A.pre = net->kpre;
    conv16_kernel<E_GATE_PRE><<<G.tiles, kCT, conv16_smem(G), s>>>(A);
    A.in = net->k1;
    A.w = net->d.k1t;
    A.u = net->u;
    convout_kernel<E_OUT_U><<<convout_grid<E_OUT_U>(G), kCT, convout_smem(G), s>>>(A);
    // loss: v = u - e_hat, w = A_hat v
    loss_prep_kernel<<<vg, kVT, 0, s>>>(T);
    spmv_store_kernel<<<h->sell_grid, kSellThreads, 0, s>>>(sell_of(h), net->t, net->y);
    loss_kernel<<<vg, kVT, 0, s>>>(T);
    // backward
    WgArgs W{};
    W.G = G;
    W.part = net->part;
    W.bias_off = -1;
    // u = C1^T(k1): dk1 = C1(du); dk = g dk1, dg = k dk1; dW1 += wgrad(k1, du)
    A.in = net->du;
    A.w = net->d.k1in;
    A.out = net->dk;
    A.pre = net->kpre;
    A.dg = net->dg;
    A.dg_add = 0;
    conv1_kernel<E_BWD_GATE><<<G.tiles, kCT, conv1_smem(G), s>>>(A);
    W.dy = net->k1;
    W.x = net->du;
    W.off = kOffW1;
    W.add = 0;
    wgrad1_kernel<<<net->wg_ctas, kCT, wgrad1_smem(G), s>>>(W);
    // k = C2^T(h2): dh2 = C2(dk); dW2 += wgrad(h2, dk)
    A.in = net->dk;
    A.w = net->d.k2;
    A.out = net->dh2;
    conv16_kernel<E_STORE><<<G.tiles, kCT, conv16_smem(G), s>>>(A);
    W.dy = net->h2;
    W.x = net->dk;
    W.off = kOffW2;
    W.add = 0;
    wgrad16_kernel<<<net->wg_ctas, kCT, wgrad16_smem(G), s>>>(W);
    // h2 = C2(h1): dW2 += wgrad(dh2, h1); dh1 = C2^T(dh2); da1 = g dh1, dg += a1 dh1
    W.dy = net->dh2;
    W.x = net->h1;
    W.add = 1;
    wgrad16_kernel<<<net->wg_ctas, kCT, wgrad16_smem(G), s>>>(W);
    A.in = net->dh2;
    A.w = net->d.k2t;
    A.out = net->da1;
    A.pre = net->a1;
    A.dg_add = 1;
    conv16_kernel<E_BWD_GATE><<<G.tiles, kCT, conv16_smem(G), s>>>(A);
    // a1 = C1(s_hat): dW1 += wgrad(da1, s_hat)
    W.dy = net->da1;
    W.x = net->shat;
    W.off = kOffW1;
    W.add = 1;
    wgrad1_kernel<<<net->wg_ctas, kCT, wgrad1_smem(G), s>>>(W);
    // gates: dag = dg g (1 - g); dWg = wgrad(dag, lognu / 8), dbg = sum dag
    const long long cnt = (long long)act_count(G, kCh);
    gate_grad_kernel<<<4 * sm_count(net->device), kVT, 0, s>>>(cnt, net->dg, L->gates, net->dag);
    W.dy = net->dag;
    W.x = L->lognu_in;
    W.off = kOffWg;
    W.bias_off = kOffBg;
    W.add = 0;
    wgrad1_kernel<<<net->wg_ctas, kCT, wgrad1_smem(G), s>>>(W);
    grad_reduce_kernel<<<(CG_LEARN_PARAMS + kVT - 1) / kVT, kVT, 0, s>>>(net->part, net->wg_ctas, net->d.grad);
}

int check_set(const cg_net *net, const cg_learn_set *set) {
    if (!net || !set || set->ninst < 1 || !set->inst || set->npairs < 1 || !set->pair_inst || !set->r || !set->e)
        return CG_EINVAL;
    const cg_handle *h0 = set->inst[0];
    if (!h0 || !h0->learn) return CG_EINVAL;
    for (int i = 0; i < set->ninst; ++i) {
        const cg_handle *h = set->inst[i];
        if (!h || !h->learn || h->device != net->device) return CG_EINVAL;
        const Geo &G = h->learn->G, &G0 = h0->learn->G;
        if (G.nx != G0.nx || G.ny != G0.ny || G.nz != G0.nz) return CG_EINVAL;
    }
    for (int64_t k = 0; k < set->npairs; ++k)
        if (set->pair_inst[k] < 0 || set->pair_inst[k] >= set->ninst) return CG_EINVAL;
    return CG_OK;
}

int max_ctas(const cg_learn_set *set) {
    int m = 1;
    for (int i = 0; i < set->ninst; ++i) m = std::max(m, set->inst[i]->ctas);
    return m;
}

}  // namespace

long long gbcg::bounds_faults_learn() { return read_bounds_faults(); }

void gbcg::learn_free(cg_handle *h) {
    if (h && h->learn) {
        free_ctx(h->learn);
        h->learn = nullptr;
    }
}

int gbcg::learn_solve(cg_handle *h, const double *b, double *x, double tol, int32_t maxit, cg_info *info) {
    LearnCtx *L = h->learn;
    if (!L || !L->net) return CG_EINVAL;
    cg_net *net = L->net;
    cudaStream_t s = h->stream;
    const size_t bytes = sizeof(double) * (size_t)h->n;
    int rc = set_smem_limits();
    if (rc != CG_OK) return rc;
    if (L->graph_net != net || !L->graph) {
        if ((rc = capture(h, L)) != CG_OK) return rc;
    }
    // the network's parameters may change between solves (training): make the
    // net's stream's work visible first
    if (cudaStreamSynchronize(net->stream) != cudaSuccess) return CG_ECUDA;
    FcgState init{};
    init.b = b;
    init.x = h->x_dev;
    init.tol = tol;
    init.n = h->n;
    init.maxit = maxit;
    init.window = L->window;
    init.factor = L->factor;
    init.reverted_at = -1;
    *L->st_host = init;
    cudaError_t e = cudaMemcpyAsync(h->x_dev, x, bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(L->st, L->st_host, sizeof(FcgState), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(L->dst, 0, sizeof(DevStatus), s);
    if (e == cudaSuccess) e = cudaEventRecord(L->t0, s);
    if (e != cudaSuccess) return CG_ECUDA;
    int launches = 0;
    launch_gates(L, net, s);
    fcg_spmv_kernel<S_SETUP><<<h->ctas, kThreads, kSmemBytes, s>>>(learn_params(h, L), L->st, h->x_dev,
                                                                   L->partials, vec_args(h, L));
    launches += 2;
    if (cudaGetLastError() != cudaSuccess) return CG_ECUDA;
    // graph launches, two in flight; each body advances the iteration count
    // by one until the solve is done, so maxit / kUnroll + 2 launches suffice
    const int max_launch = maxit / kUnroll + 2;
    int launched = 0, waited = 0;
    bool stop = false;
    while (!stop) {
        while (launched - waited < 2 && launched < max_launch) {
            const int sl = launched & 1;
            e = cudaGraphLaunch(L->graph, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(&L->flags_host[sl], &L->st->n, sizeof(FcgFlags), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(&L->dst_host[sl], L->dst, sizeof(DevStatus), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaEventRecord(L->ev[sl], s);
            if (e != cudaSuccess) return CG_ECUDA;
            ++launched;
            launches += body_kernels(L) * kUnroll;
        }
        if (waited == launched) break;
        const int sl = waited & 1;
        if (cudaEventSynchronize(L->ev[sl]) != cudaSuccess) return CG_ECUDA;
        ++waited;
        const FcgFlags f = L->flags_host[sl];
        if (f.done || L->dst_host[sl].status != 0) stop = true;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return CG_ECUDA;
    if (h->opts.true_residual) {
        fcg_spmv_kernel<S_TRUE><<<h->ctas, kThreads, kSmemBytes, s>>>(learn_params(h, L), L->st, h->x_dev,
                                                                      L->partials, vec_args(h, L));
        ++launches;
    }
    e = cudaEventRecord(L->t1, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(L->st_host, L->st, sizeof(FcgState), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(L->dst_host, L->dst, sizeof(DevStatus), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return CG_ECUDA;
    const FcgState &st = *L->st_host;
    int status = L->dst_host[0].status != 0 ? L->dst_host[0].status : (st.done ? st.status : CG_ENOCONV);
    if (st.bb == 0.0 && status == CG_OK) {
        if (cudaMemsetAsync(h->x_dev, 0, bytes, s) != cudaSuccess) return CG_ECUDA;
    }
    if (cudaMemcpyAsync(x, h->x_dev, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return CG_ECUDA;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, L->t0, L->t1);
    if (info) {
        cg_info out{};
        out.iters = st.iters;
        out.status = status;
        out.relres = st.bnorm > 0.0 ? std::sqrt(st.rr) / st.bnorm : 0.0;
        out.relres_true = (!h->opts.true_residual || status == CG_ENAN) ? -1.0
                          : (st.bnorm > 0.0 ? std::sqrt(std::max(st.true_rr, 0.0)) / st.bnorm : 0.0);
        out.kernel_ms = ms;
        out.launches = launches;
        out.outer = 0;
        out.reverted_at = st.reverted_at;
        *info = out;
    }
    return status;
}

extern "C" {

int cg_net_create(const float *params, cg_net **out) {
    if (!out) return CG_EINVAL;
    *out = nullptr;
    if (!params || !finite_params(params)) return CG_EINVAL;
    cg_net *net = new (std::nothrow) cg_net();
    if (!net) return CG_ENOMEM;
    if (cudaGetDevice(&net->device) != cudaSuccess) {
        delete net;
        return CG_ECUDA;
    }
    auto fail = [&](int rc) {
        cg_net_destroy(net);
        return rc;
    };
    if (cudaStreamCreateWithFlags(&net->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(CG_ECUDA);
    const size_t P = CG_LEARN_PARAMS;
    const size_t sizes[] = {P * 4, P * 4, P * 4, P * 4, kCh * kTapsPad * 2, kTaps * kCh * 2, kTaps * kCh * kCh * 2,
                            kTaps * kCh * kCh * 2, kCh * kTapsPad * 2, kCh * 4, 8 * 4096};
    size_t offs[11], total = 0;
    for (int i = 0; i < 11; ++i) {
        offs[i] = total;
        total += (sizes[i] + 255) / 256 * 256;
    }
    if (cudaMalloc(&net->block, total) != cudaSuccess) return fail(CG_ENOMEM);
    if (cudaMemset(net->block, 0, total) != cudaSuccess) return fail(CG_ECUDA);
    char *b = static_cast<char *>(net->block);
    net->d.theta = reinterpret_cast<float *>(b + offs[0]);
    net->d.m = reinterpret_cast<float *>(b + offs[1]);
    net->d.v = reinterpret_cast<float *>(b + offs[2]);
    net->d.grad = reinterpret_cast<float *>(b + offs[3]);
    net->d.k1in = reinterpret_cast<__nv_bfloat16 *>(b + offs[4]);
    net->d.k1t = reinterpret_cast<__nv_bfloat16 *>(b + offs[5]);
    net->d.k2 = reinterpret_cast<__nv_bfloat16 *>(b + offs[6]);
    net->d.k2t = reinterpret_cast<__nv_bfloat16 *>(b + offs[7]);
    net->d.kgin = reinterpret_cast<__nv_bfloat16 *>(b + offs[8]);
    net->d.bg = reinterpret_cast<float *>(b + offs[9]);
    net->d.loss_hist = reinterpret_cast<double *>(b + offs[10]);
    net->loss_cap_n = 4096;
    int rc = upload_params(net, params);
    if (rc != CG_OK) return fail(rc);
    *out = net;
    return CG_OK;
}

int cg_net_get_params(const cg_net *net, float *params) {
    if (!net || !params) return CG_EINVAL;
    DeviceGuard g(net->device);
    if (cudaStreamSynchronize(net->stream) != cudaSuccess ||
        cudaMemcpy(params, net->d.theta, sizeof(float) * CG_LEARN_PARAMS, cudaMemcpyDeviceToHost) != cudaSuccess)
        return CG_ECUDA;
    return CG_OK;
}

int cg_net_set_params(cg_net *net, const float *params) {
    if (!net || !params || !finite_params(params)) return CG_EINVAL;
    DeviceGuard g(net->device);
    return upload_params(net, params);
}

void cg_net_destroy(cg_net *net) {
    if (!net) return;
    DeviceGuard g(net->device);
    if (net->stream) cudaStreamSynchronize(net->stream);
    for (void *p : net->tallocs) cudaFree(p);
    if (net->block) cudaFree(net->block);
    if (net->stream) cudaStreamDestroy(net->stream);
    delete net;
}

int cg_set_learned(cg_handle *h, cg_net *net, int32_t ex, int32_t ey, int32_t ez, const float *lognu,
                   int32_t stall_window, double stall_factor) {
    NvtxRange nvtx("gbcg.set_learned");
    if (!h || !net || !lognu || h->opts.precond != CG_PRECOND_LEARNED) return CG_EINVAL;
    if (ex < 1 || ey < 1 || ez < 1) return CG_EINVAL;
    if ((int64_t)(ex + 1) * (ey + 1) * (ez + 1) != (int64_t)h->n) return CG_EINVAL;
    if (stall_window == 0) stall_window = 50;
    if (stall_factor == 0.0) stall_factor = 0.9;
    if (stall_window < 1 || stall_window > kMaxWindow || !(stall_factor > 0.0 && stall_factor <= 1.0))
        return CG_EINVAL;
    if (net->device != h->device) return CG_EINVAL;
    for (int32_t i = 0; i < h->n; ++i)
        if (!std::isfinite(lognu[i])) return CG_EINVAL;
    DeviceGuard dg(h->device);
    int rc = set_smem_limits();
    if (rc != CG_OK) return rc;
    learn_free(h);
    LearnCtx *L = new (std::nothrow) LearnCtx();
    if (!L) return CG_ENOMEM;
    auto fail = [&](int code) {
        free_ctx(L);
        return code;
    };
    L->net = net;
    L->G = make_geo(ex, ey, ez);
    L->window = stall_window;
    L->factor = stall_factor;
    const Geo &G = L->G;
    const int sms = sm_count(h->device);
    L->vgrid = std::min((G.n + kVT - 1) / kVT, 4 * sms);
    // the fused SELL-32 kernel needs the handle's SELL-32 CTA ranges (every
    // handle whose FP64 solve runs a SELL-32 kernel) and one resident CTA of
    // 1024 threads per SM
    if (h->sell_cut) {
        int occ = 0;
        if (cudaFuncSetAttribute((const void *)fcg_sell_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxL1) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fcg_sell_kernel, kSellSolveThreads, 0) !=
                cudaSuccess)
            return fail(CG_ECUDA);
        L->fused = occ >= 1 && h->ctas <= occ * sms;
    }
    const size_t a16 = act_count(G, kCh);
    auto &A = L->allocs;
    const int nparts = std::max({L->vgrid, G.tiles, h->ctas, h->sell_grid});
    if ((rc = ctx_alloc(A, &L->lognu_in, act_count(G, 1))) || (rc = ctx_alloc(A, &L->gates, a16)) ||
        (rc = ctx_alloc(A, &L->s_in, act_count(G, 1))) || (rc = ctx_alloc(A, &L->pidx, (size_t)G.n)) ||
        (rc = ctx_alloc(A, &L->h1, a16)) || (rc = ctx_alloc(A, &L->h2, a16)) || (rc = ctx_alloc(A, &L->k1, a16)) ||
        (rc = ctx_alloc(A, &L->dsq, (size_t)G.n)) || (rc = ctx_alloc(A, &L->r, (size_t)G.n)) ||
        (rc = ctx_alloc(A, &L->z, (size_t)G.n + 16)) || (rc = ctx_alloc(A, &L->p, (size_t)G.n + 16)) ||
        (rc = ctx_alloc(A, &L->dsq32, (size_t)G.n)) ||
        (rc = ctx_alloc(A, &L->q, (size_t)G.n)) || (rc = ctx_alloc(A, &L->partials, (size_t)3 * nparts)) ||
        (rc = ctx_alloc(A, &L->sigma, 4)) || (rc = ctx_alloc(A, &L->counter, 4)) || (rc = ctx_alloc(A, &L->st, 1)) ||
        (rc = ctx_alloc(A, &L->dst, 1)) || (rc = ctx_alloc(A, &L->conv_err, 1)))
        return fail(rc);
    if (cudaMallocHost(&L->st_host, sizeof(FcgState)) != cudaSuccess ||
        cudaMallocHost(&L->flags_host, 2 * sizeof(FcgFlags)) != cudaSuccess ||
        cudaMallocHost(&L->dst_host, 2 * sizeof(DevStatus)) != cudaSuccess)
        return fail(CG_ENOMEM);
    if (cudaStreamCreateWithFlags(&L->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&L->ev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&L->ev[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&L->t0) != cudaSuccess || cudaEventCreate(&L->t1) != cudaSuccess)
        return fail(CG_ECUDA);
    // log nu / 8 into the padded one-channel field (BF16)
    std::vector<uint16_t> ln((size_t)(G.npad + kSlack), 0);
    std::vector<int32_t> pidx((size_t)G.n);
    for (int32_t i = 0; i < G.n; ++i) {
        const int x = i % G.nx, rest = i / G.nx, y = rest % G.ny, z = rest / G.ny;
        const size_t pos = (size_t)(z + 1) * G.plane + (size_t)(y + 1) * G.px + (x + 1);
        ln[pos] = bf16_bits_rne((double)lognu[i] * kLogNuScale);
        pidx[i] = (int32_t)pos;
    }
    if (cudaMemcpy(L->lognu_in, ln.data(), ln.size() * 2, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(L->pidx, pidx.data(), pidx.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(CG_ECUDA);
    dsq_kernel<<<L->vgrid, kVT, 0, h->stream>>>(G.n, h->dinv, L->dsq, L->dsq32);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(h->stream) != cudaSuccess) return fail(CG_ECUDA);
    h->learn = L;
    return CG_OK;
}

int cg_precond_apply(cg_handle *h, const double *r, double *z) {
    NvtxRange nvtx("gbcg.precond_apply");
    if (!h || !h->learn || !r || !z) return CG_EINVAL;
    LearnCtx *L = h->learn;
    DeviceGuard dg(h->device);
    int rc = set_smem_limits();
    if (rc != CG_OK) return rc;
    if (cudaStreamSynchronize(L->net->stream) != cudaSuccess) return CG_ECUDA;
    const Geo &G = L->G;
    cudaStream_t s = h->stream;
    launch_gates(L, L->net, s);
    sigma_kernel<double><<<L->vgrid, kVT, 0, s>>>(G.n, r, h->dinv, L->sigma, L->counter, L->partials);
    scatter_s_kernel<<<L->vgrid, kVT, 0, s>>>(G.n, r, L->dsq, L->pidx, L->s_in);
    ConvArgs A = conv_args(G);
    A.dsq = L->dsq;
    A.dsq32 = L->dsq32;
    A.gate = L->gates;
    A.sigma = L->sigma;
    A.in = L->s_in;
    A.w = L->net->d.k1in;
    A.out = L->h1;
    conv1_kernel<E_GATE><<<G.tiles, kCT, conv1_smem(G), s>>>(A);
    A.in = L->h1;
    A.w = L->net->d.k2;
    A.out = L->h2;
    A.wait_ns = (unsigned long long)(h->opts.wait_limit_s * 1e9);
    A.err = L->conv_err;
    conv16tc_kernel<E_STORE><<<G.ttiles, kCT, conv16tc_smem(G), s>>>(A);
    A.in = L->h2;
    A.w = L->net->d.k2t;
    A.out = L->k1;
    conv16tc_kernel<E_GATE><<<G.ttiles, kCT, conv16tc_smem(G), s>>>(A);
    A.in = L->k1;
    A.w = L->net->d.k1t;
    A.z = z;
    convout_kernel<E_OUT_Z><<<convout_grid<E_OUT_Z>(G), kCT, convout_smem(G), s>>>(A);
    int err = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&err, L->conv_err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return CG_ECUDA;
    return err ? err : CG_OK;
}

int cg_learn_pairs(cg_handle *h, const double *b, const double *xstar, int32_t segment, int32_t count,
                   float *r_out, float *e_out) {
    NvtxRange nvtx("gbcg.learn_pairs");
    if (!h || !h->learn || !b || !xstar || !r_out || !e_out || segment < 1 || count < 1) return CG_EINVAL;
    DeviceGuard dg(h->device);
    LearnCtx *L = h->learn;
    cudaStream_t s = h->stream;
    const int n = h->n;
    if (cudaMemsetAsync(h->x_dev, 0, sizeof(double) * (size_t)n, s) != cudaSuccess) return CG_ECUDA;
    int rc = CG_OK;
    for (int32_t k = 0; k < count && rc == CG_OK; ++k) {
        rc = enqueue_spmv(h, h->x_dev, L->q);
        if (rc == CG_OK) {
            pair_record_kernel<<<L->vgrid, kVT, 0, s>>>(n, b, xstar, h->x_dev, L->q, r_out + (size_t)k * n,
                                                        e_out + (size_t)k * n);
            if (cudaGetLastError() != cudaSuccess) rc = CG_ECUDA;
        }
        if (rc == CG_OK && k + 1 < count) rc = enqueue_fp64_solve(h, b, h->x_dev, 0.0, segment, 0);
        if (rc == CG_OK && (k & 15) == 15 && cudaStreamSynchronize(s) != cudaSuccess) rc = CG_ECUDA;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return CG_ECUDA;
    if (rc != CG_OK) return rc;
    const int st = h->st_host->status;
    if (count > 1 && st != CG_OK && st != CG_ENOCONV) return st;
    return CG_OK;
}

int cg_learn_grad(cg_net *net, const cg_learn_set *set, const int64_t *pairs, int32_t count, double *loss,
                  float *grad) {
    NvtxRange nvtx("gbcg.learn_grad");
    int rc = check_set(net, set);
    if (rc != CG_OK) return rc;
    if (!pairs || count < 1 || !loss) return CG_EINVAL;
    for (int32_t k = 0; k < count; ++k)
        if (pairs[k] < 0 || pairs[k] >= set->npairs) return CG_EINVAL;
    DeviceGuard dg(net->device);
    if ((rc = set_smem_limits()) != CG_OK) return rc;
    const Geo &G = set->inst[0]->learn->G;
    if ((rc = ensure_train(net, G, max_ctas(set))) != CG_OK) return rc;
    for (int i = 0; i < set->ninst; ++i)
        if (cudaStreamSynchronize(set->inst[i]->stream) != cudaSuccess) return CG_ECUDA;
    cudaStream_t s = net->stream;
    if (cudaMemsetAsync(net->d.grad, 0, sizeof(float) * CG_LEARN_PARAMS, s) != cudaSuccess ||
        cudaMemsetAsync(net->scal, 0, sizeof(double) * 8, s) != cudaSuccess)
        return CG_ECUDA;
    for (int32_t k = 0; k < count; ++k) {
        const int64_t idx = pairs[k];
        cg_handle *h = set->inst[set->pair_inst[idx]];
        enqueue_sample(net, h, set->r + (size_t)idx * G.n, set->e + (size_t)idx * G.n);
    }
    if (cudaGetLastError() != cudaSuccess) return CG_ECUDA;
    std::vector<float> g(CG_LEARN_PARAMS);
    double sc[8];
    if (cudaMemcpyAsync(g.data(), net->d.grad, sizeof(float) * CG_LEARN_PARAMS, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(sc, net->scal, sizeof(sc), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemsetAsync(net->d.grad, 0, sizeof(float) * CG_LEARN_PARAMS, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return CG_ECUDA;
    *loss = sc[2] / count;
    if (grad) {
        const double scale = 1.0 / ((double)G.n * count);
        for (int j = 0; j < CG_LEARN_PARAMS; ++j) grad[j] = (float)(g[j] * scale);
    }
    return CG_OK;
}

int cg_learn_train(cg_net *net, const cg_learn_set *set, const int64_t *order, int32_t steps, int32_t batch,
                   float lr, double *losses) {
    NvtxRange nvtx("gbcg.learn_train");
    int rc = check_set(net, set);
    if (rc != CG_OK) return rc;
    if (!order || steps < 1 || batch < 1 || !(lr > 0.0f) || !std::isfinite(lr)) return CG_EINVAL;
    for (int64_t k = 0; k < (int64_t)steps * batch; ++k)
        if (order[k] < 0 || order[k] >= set->npairs) return CG_EINVAL;
    DeviceGuard dg(net->device);
    if ((rc = set_smem_limits()) != CG_OK) return rc;
    const Geo &G = set->inst[0]->learn->G;
    if ((rc = ensure_train(net, G, max_ctas(set))) != CG_OK) return rc;
    for (int i = 0; i < set->ninst; ++i)
        if (cudaStreamSynchronize(set->inst[i]->stream) != cudaSuccess) return CG_ECUDA;
    cudaStream_t s = net->stream;
    if (cudaMemsetAsync(net->d.grad, 0, sizeof(float) * CG_LEARN_PARAMS, s) != cudaSuccess ||
        cudaMemsetAsync(net->scal, 0, sizeof(double) * 8, s) != cudaSuccess)
        return CG_ECUDA;
    std::vector<double> hist;
    for (int32_t k = 0; k < steps; ++k) {
        for (int32_t j = 0; j < batch; ++j) {
            const int64_t idx = order[(int64_t)k * batch + j];
            cg_handle *h = set->inst[set->pair_inst[idx]];
            enqueue_sample(net, h, set->r + (size_t)idx * G.n, set->e + (size_t)idx * G.n);
        }
        ++net->step;
        const float bc1 = 1.0f - std::pow(0.9f, (float)net->step);
        const float bc2 = 1.0f - std::pow(0.999f, (float)net->step);
        const int slot = k % net->loss_cap_n;
        adam_kernel<<<(CG_LEARN_PARAMS + kVT - 1) / kVT, kVT, 0, s>>>(
            net->d, (float)(1.0 / ((double)G.n * batch)), lr, bc1, bc2, net->scal, 1.0 / batch, slot);
        if (cudaGetLastError() != cudaSuccess) return CG_ECUDA;
        if (slot == net->loss_cap_n - 1 || k == steps - 1) {
            std::vector<double> buf(slot + 1);
            if (cudaMemcpyAsync(buf.data(), net->d.loss_hist, sizeof(double) * (slot + 1), cudaMemcpyDeviceToHost, s) !=
                    cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                return CG_ECUDA;
            hist.insert(hist.end(), buf.begin(), buf.end());
        }
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return CG_ECUDA;
    if (losses) std::memcpy(losses, hist.data(), sizeof(double) * steps);
    return CG_OK;
}

}  // extern "C"
