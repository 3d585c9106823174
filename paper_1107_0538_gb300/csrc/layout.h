// Geometry of the SpMV tiles and shared-memory stages, shared by the host
// planner (plan.h) and the kernels (cg_device.cuh).  Plain C++.
#pragma once

#include <cstdint>

namespace gbcg {

// ---------------------------------------------------------------- geometry
// FP64 arithmetic is the scarce resource on GB300 (about 2 FP64 FMA per clock
// per SM, 56x below FP32), so the SpMV gives every row to one thread: exactly
// one FMA per stored entry, no cross-lane reduction adds, no padded slots.
// Each warp streams its own tiles of up to 32 rows (one per lane) through a
// shared-memory stage of its own with TMA bulk copies and its own mbarrier,
// so warps never wait for each other inside the SpMV.  A stage holds the
// tile's values, its column indices, its row pointers and, for "windowed"
// tiles, the x-window: the few contiguous segments of the multiplied vector
// that the tile's columns touch (9 to 12 segments for a 27-point stencil).
// The column indices of a windowed tile are 16-bit offsets into that window,
// so every gather of the product is a shared-memory read.
constexpr int kThreads = 512;                  // threads per CTA
constexpr int kWarps = kThreads / 32;
constexpr int kTileRows = 32;                  // rows per warp tile (one per lane)
constexpr int kTileNnz = 864;                  // stored entries per warp tile (32 rows x 27)
constexpr int kWinMax = 440;                   // elements of x-window per tile
constexpr int kSegAlign = 4;                   // window segments start/end on 4 elements:
                                               // 16-byte TMA alignment for FP64 and FP32 vectors
constexpr int kSegMax = 32;                    // window segments per tile (one per lane)
constexpr int kBatch = 9;                      // loads in flight per thread
constexpr int kValsStage = kTileNnz + 8;       // doubles per stage (alignment slack)
constexpr int kColsStage = kTileNnz + 8;       // int32 (or 2x uint16) per stage
constexpr int kRptrStage = kTileRows + 8;      // int32 per stage (row pointers)
constexpr int kStageBytes = 14208;             // holds every layout below

// Offsets inside a stage for stored values of VB bytes and vector elements of
// XB bytes: values, column indices (int32, or uint16 for windowed tiles), row
// pointers, x-window.
template <int VB, int XB>
struct StageLayout {
    static constexpr int vals_off = 0;
    static constexpr int cols_off = ((kValsStage * VB + 15) / 16) * 16;
    static constexpr int rptr_off = cols_off + kColsStage * 4;
    static constexpr int win_off = rptr_off + kRptrStage * 4;
    static constexpr int end = win_off + kWinMax * XB;
    static_assert(end <= kStageBytes, "stage too small for this value/vector type");
    static_assert(cols_off % 16 == 0 && rptr_off % 16 == 0 && win_off % 16 == 0, "stage alignment");
};
constexpr int kRedSlots = 4;                   // partial sums per CTA per barrier
constexpr int kSmemBytes = kWarps * kStageBytes + kWarps * 8 /*mbarriers*/ +
                           kThreads * 8 /*block-sum transpose*/ + 64 /*broadcast*/ + 64 /*control*/;
constexpr int kMaxRegRows = 4;                 // largest rows-per-thread kept in registers
static_assert(kStageBytes % 16 == 0, "stage alignment");
static_assert(kTileNnz + 6 <= kColsStage && kTileNnz + 2 <= kValsStage, "stage slack");
static_assert(kTileRows + 1 + 6 <= kRptrStage, "row pointer slack");
static_assert(kSmemBytes <= 232448, "shared memory per CTA");

// Kinds of tile.
constexpr int kTileWindow = 0;   // 16-bit local columns into a staged x-window
constexpr int kTileGather = 1;   // 32-bit global columns, gathers from global memory
constexpr int kTileLong = 2;     // one row longer than kTileNnz, read from global memory

// One row tile: rows [r0, r1) holding entries [a, e); window segments
// segs[seg0 .. seg0 + nseg) whose TMA copies deliver wtx elements in total.
struct TileDesc {
    int32_t r0, r1, a, e;
    int32_t seg0, nseg, wtx, kind;
};

}  // namespace gbcg
