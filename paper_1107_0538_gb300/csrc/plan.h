// Host-side planning of the SpMV tiles (plain C++, no CUDA calls): row
// tiles, their x-windows and 16-bit local columns, the split of tiles over
// CTAs, and a checker of every index the kernels derive from the plan.
#pragma once

#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "layout.h"

namespace gbcg {

struct I4 {
    int32_t x, y, z, w;
};
inline I4 mk4(int32_t x, int32_t y, int32_t z, int32_t w) { return I4{x, y, z, w}; }

// Row tiles: at most kTileRows rows and kTileNnz entries each; a row with
// more than kTileNnz entries is a tile of its own (read from global memory).
inline std::vector<int32_t> plan_tiles(int32_t n, const std::vector<int32_t> &rowptr, int *max_nnz) {
    std::vector<int32_t> tiles;
    tiles.reserve(n / 16 + 2);
    int32_t r = 0;
    *max_nnz = 0;
    while (r < n) {
        const int32_t start = r;
        if (rowptr[r + 1] - rowptr[r] > kTileNnz) {
            ++r;
        } else {
            while (r < n && r - start < kTileRows && rowptr[r + 1] - rowptr[r] <= kTileNnz &&
                   rowptr[r + 1] - rowptr[start] <= kTileNnz)
                ++r;
        }
        tiles.push_back(start);
        *max_nnz = std::max(*max_nnz, rowptr[r] - rowptr[start]);
    }
    tiles.push_back(n);
    return tiles;
}

// x-window of one tile: the distinct columns grouped into runs (gaps of up
// to kGap unused columns are bridged), each run widened to kSegAlign-element
// boundaries so that its TMA copy is 16-byte aligned for FP64 and FP32
// vectors alike.  A run that would end past the vector's last column stops
// at the last aligned column n & ~3; the 1 to 3 columns after it (its tail)
// are stored into the window by threads.  Windowed when the runs fit kSegMax
// lanes and kWinMax elements; each entry then stores its 16-bit offset in
// the window.
constexpr int kGap = 4;

struct TilePlan {
    std::vector<I4> desc;       // 2 per tile
    std::vector<I4> segs;
    std::vector<uint16_t> lcol;   // nnz (+ padding)
    int windowed = 0;
};

inline TilePlan plan_windows(int32_t n, const std::vector<int32_t> &rowptr, const std::vector<int32_t> &colidx,
                      const std::vector<int32_t> &tiles) {
    TilePlan tp;
    const int nt = (int)tiles.size() - 1;
    tp.desc.resize(2 * (size_t)std::max(nt, 1), mk4(0, 0, 0, 0));
    tp.lcol.assign(colidx.size() + 32, 0);
    std::vector<int32_t> cols;
    std::vector<I4> runs;
    for (int t = 0; t < nt; ++t) {
        const int r0 = tiles[t], r1 = tiles[t + 1];
        const int a = rowptr[r0], e = rowptr[r1];
        int kind = kTileGather, seg0 = 0, nseg = 0, wtx = 0;
        if (e - a > kTileNnz) {
            kind = kTileLong;
        } else if (e > a) {
            cols.assign(colidx.begin() + a, colidx.begin() + e);
            std::sort(cols.begin(), cols.end());
            cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
            // runs [first, last] of columns, bridged over small gaps, aligned
            runs.clear();
            int first = cols[0], last = cols[0];
            auto flush = [&]() {
                const int gs = first & ~(kSegAlign - 1);
                int ge = (last + kSegAlign) & ~(kSegAlign - 1);  // exclusive, aligned
                if (!runs.empty() && gs <= runs.back().y) {
                    runs.back().y = std::max(runs.back().y, ge);
                } else {
                    runs.push_back(mk4(gs, ge, 0, 0));
                }
            };
            for (size_t i = 1; i < cols.size(); ++i) {
                if (cols[i] - last <= kGap + 1) {
                    last = cols[i];
                } else {
                    flush();
                    first = last = cols[i];
                }
            }
            flush();
            // window layout
            int woff = 0, tx = 0;
            std::vector<I4> segs;
            for (const I4 &rr : runs) {
                I4 sg;
                sg.x = rr.x;
                sg.y = woff;
                if (rr.y > n) {  // runs past the vector: copy up to n & ~3, store the tail
                    sg.z = (n & ~(kSegAlign - 1)) - rr.x;
                    sg.w = n & ~(kSegAlign - 1);
                } else {
                    sg.z = rr.y - rr.x;
                    sg.w = -1;
                }
                woff += rr.y - rr.x;
                tx += sg.z;
                segs.push_back(sg);
            }
            if ((int)segs.size() <= kSegMax && woff <= kWinMax) {
                kind = kTileWindow;
                seg0 = (int)tp.segs.size();
                nseg = (int)segs.size();
                wtx = tx;
                tp.segs.insert(tp.segs.end(), segs.begin(), segs.end());
                for (int k = a; k < e; ++k) {
                    const int c = colidx[k];
                    // the run holding c (runs are sorted and disjoint)
                    int lo = 0, hi = nseg - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) / 2;
                        if (segs[mid].x <= c) lo = mid;
                        else hi = mid - 1;
                    }
                    tp.lcol[k] = (uint16_t)(segs[lo].y + (c - segs[lo].x));
                }
                ++tp.windowed;
            }
        }
        tp.desc[2 * t] = mk4(r0, r1, a, e);
        tp.desc[2 * t + 1] = mk4(seg0, nseg, wtx, kind);
    }
    if (tp.segs.empty()) tp.segs.push_back(mk4(0, 0, 0, -1));
    return tp;
}

// Contiguous tile ranges per CTA with about equal cost (entries + rows).
inline std::vector<int32_t> split_tiles(const std::vector<int32_t> &tiles, const std::vector<int32_t> &rowptr,
                                 int ctas) {
    const int nt = (int)tiles.size() - 1;
    std::vector<double> prefix(nt + 1, 0.0);
    for (int t = 0; t < nt; ++t) {
        const double nnz = rowptr[tiles[t + 1]] - rowptr[tiles[t]];
        const double rows = tiles[t + 1] - tiles[t];
        prefix[t + 1] = prefix[t] + nnz + 2.0 * rows;
    }
    std::vector<int32_t> cut(ctas + 1, 0);
    int t = 0;
    for (int b = 1; b < ctas; ++b) {
        const double target = prefix[nt] * b / ctas;
        while (t < nt && prefix[t + 1] <= target) ++t;
        // choose the boundary closer to the target
        if (t < nt && target - prefix[t] > prefix[t + 1] - target) ++t;
        cut[b] = std::max(cut[b - 1], t);
    }
    cut[ctas] = nt;
    return cut;
}


// Batch of independent systems laid out as one block-diagonal matrix: row
// tiles never cross a system boundary, each tile knows its system, and every
// (CTA, system) pair with tiles on that CTA is a reduction segment.  Segments
// are ordered by CTA and by system at once, so each CTA owns a contiguous run
// of segments and so does each system.
struct BatchPlan {
    std::vector<int32_t> tiles;        // row boundaries (ntiles + 1)
    std::vector<int32_t> tile_sys;     // system of each tile
    std::vector<int32_t> cut;          // CTA -> tile range (ctas + 1)
    std::vector<int32_t> cta_sys0;     // first system of each CTA (ctas + 1; last = nsys)
    std::vector<int32_t> cta_nsys;     // systems of each CTA
    std::vector<int32_t> cta_seg0;     // first segment of each CTA (ctas + 1)
    std::vector<int32_t> sys_seg0;     // first segment of each system (nsys + 1)
    std::vector<int32_t> sys_cta0;     // first CTA holding each system
    std::vector<int32_t> seg_cta;      // CTA of each segment
    int max_nsys_per_cta = 0;
};

inline BatchPlan plan_batch(const std::vector<int32_t> &rowptr, const std::vector<int32_t> &sys_rows,
                            int ctas, int *max_tile_nnz) {
    BatchPlan bp;
    const int nsys = (int)sys_rows.size() - 1;
    *max_tile_nnz = 0;
    for (int s = 0; s < nsys; ++s) {
        const int r0 = sys_rows[s], r1 = sys_rows[s + 1];
        int r = r0;
        while (r < r1) {
            const int start = r;
            if (rowptr[r + 1] - rowptr[r] > kTileNnz) {
                ++r;
            } else {
                while (r < r1 && r - start < kTileRows && rowptr[r + 1] - rowptr[r] <= kTileNnz &&
                       rowptr[r + 1] - rowptr[start] <= kTileNnz)
                    ++r;
            }
            bp.tiles.push_back(start);
            bp.tile_sys.push_back(s);
            *max_tile_nnz = std::max(*max_tile_nnz, rowptr[r] - rowptr[start]);
        }
    }
    bp.tiles.push_back(sys_rows[nsys]);
    const int nt = (int)bp.tile_sys.size();
    bp.cut = split_tiles(bp.tiles, rowptr, ctas);
    bp.cta_sys0.assign(ctas + 1, 0);
    bp.cta_nsys.assign(ctas, 0);
    bp.cta_seg0.assign(ctas + 1, 0);
    bp.sys_seg0.assign(nsys + 1, 0);
    bp.sys_cta0.assign(nsys, -1);
    std::vector<int32_t> seg_sys;
    for (int c = 0; c < ctas; ++c) {
        bp.cta_seg0[c] = (int)seg_sys.size();
        const int t0 = bp.cut[c], t1 = bp.cut[c + 1];
        if (t1 <= t0) continue;
        const int s0 = bp.tile_sys[t0], s1 = bp.tile_sys[t1 - 1];
        bp.cta_sys0[c] = s0;
        bp.cta_nsys[c] = s1 - s0 + 1;
        for (int s = s0; s <= s1; ++s) {
            if (bp.sys_cta0[s] < 0) bp.sys_cta0[s] = c;
            bp.seg_cta.push_back(c);
            seg_sys.push_back(s);
        }
        bp.max_nsys_per_cta = std::max(bp.max_nsys_per_cta, s1 - s0 + 1);
    }
    bp.cta_seg0[ctas] = (int)seg_sys.size();
    bp.cta_sys0[ctas] = nsys;
    // the segments of each system follow each other (seg_sys never decreases)
    for (int s = 0; s <= nsys; ++s)
        bp.sys_seg0[s] = (int)(std::lower_bound(seg_sys.begin(), seg_sys.end(), s) - seg_sys.begin());
    (void)nt;
    return bp;
}

// Checks the batch plan: tiles inside one system, CTA system ranges and
// segments consistent in both orders.  Empty string when sound.
inline std::string check_batch_plan(const BatchPlan &bp, const std::vector<int32_t> &sys_rows, int ctas) {
    const int nsys = (int)sys_rows.size() - 1;
    const int nt = (int)bp.tile_sys.size();
    for (int t = 0; t < nt; ++t) {
        const int s = bp.tile_sys[t];
        if (s < 0 || s >= nsys || bp.tiles[t] < sys_rows[s] || bp.tiles[t + 1] > sys_rows[s + 1])
            return "tile " + std::to_string(t) + " crosses a system";
    }
    int k = 0;
    for (int c = 0; c < ctas; ++c) {
        if (bp.cta_seg0[c] != k) return "cta segment start";
        for (int j = 0; j < bp.cta_nsys[c]; ++j, ++k) {
            const int s = bp.cta_sys0[c] + j;
            if (k >= (int)bp.seg_cta.size() || bp.seg_cta[k] != c) return "segment cta";
            if (k < bp.sys_seg0[s] || k >= bp.sys_seg0[s + 1]) return "segment outside its system run";
        }
        for (int t = bp.cut[c]; t < bp.cut[c + 1]; ++t) {
            const int s = bp.tile_sys[t];
            if (s < bp.cta_sys0[c] || s >= bp.cta_sys0[c] + bp.cta_nsys[c]) return "tile system outside cta range";
        }
    }
    for (int s = 0; s < nsys; ++s) {
        for (int q = bp.sys_seg0[s]; q < bp.sys_seg0[s + 1]; ++q) {
            const int c = bp.seg_cta[q];
            if (s < bp.cta_sys0[c] || s >= bp.cta_sys0[c] + bp.cta_nsys[c]) return "system segment on wrong cta";
        }
        if (sys_rows[s + 1] > sys_rows[s] && bp.sys_seg0[s + 1] <= bp.sys_seg0[s]) return "system without segments";
    }
    return std::string();
}

// Checks every address the kernels form from a plan: TMA source ranges inside
// the (padded) arrays, copy sizes inside the stage regions, window segments
// aligned and inside [0, n), and each windowed entry's local column pointing
// back at its global column.  Returns an empty string when the plan is sound.
inline std::string check_plan(int32_t n, const std::vector<int32_t> &rowptr,
                              const std::vector<int32_t> &colidx, const std::vector<int32_t> &tiles,
                              const TilePlan &tp, int64_t pad) {
    const int64_t nnz = (int64_t)colidx.size();
    const int nt = (int)tiles.size() - 1;
    auto err = [](int t, const char *what) { return "tile " + std::to_string(t) + ": " + what; };
    for (int t = 0; t < nt; ++t) {
        const I4 d0 = tp.desc[2 * t], d1 = tp.desc[2 * t + 1];
        const int r0 = d0.x, r1 = d0.y, a = d0.z, e = d0.w, seg0 = d1.x, nseg = d1.y, wtx = d1.z, kind = d1.w;
        if (r0 != tiles[t] || r1 != tiles[t + 1] || a != rowptr[r0] || e != rowptr[r1]) return err(t, "descriptor");
        if (r1 <= r0 || r1 - r0 > kTileRows) return err(t, "rows");
        if (kind == kTileLong) {
            if (r1 - r0 != 1 || e - a <= kTileNnz) return err(t, "long row");
            continue;
        }
        if (e - a > kTileNnz) return err(t, "entries");
        const int ra = r0 & ~3, re = (r1 + 1 + 3) & ~3;
        if (ra < 0 || re > n + 1 + pad || re - ra > kRptrStage) return err(t, "row pointer copy");
        if (e > a) {
            const int va = a & ~1, ve = (e + 1) & ~1;
            if (va < 0 || ve > nnz + pad || ve - va > kValsStage) return err(t, "value copy");
            if (kind == kTileWindow) {
                const int ca = a & ~7, ce = (e + 7) & ~7;
                if (ca < 0 || ce > nnz + 32 || (ce - ca) * 2 > kColsStage * 4) return err(t, "local column copy");
            } else {
                const int ca = a & ~3, ce = (e + 3) & ~3;
                if (ca < 0 || ce > nnz + pad || ce - ca > kColsStage) return err(t, "column copy");
            }
        }
        if (kind != kTileWindow) {
            if (nseg != 0 || wtx != 0) return err(t, "window on a gather tile");
            continue;
        }
        if (nseg < 1 || nseg > kSegMax || seg0 < 0 || seg0 + nseg > (int)tp.segs.size()) return err(t, "segments");
        int tx = 0, slots_end = 0;
        for (int i = 0; i < nseg; ++i) {
            const I4 sg = tp.segs[seg0 + i];
            const int al = kSegAlign - 1;
            if (sg.x < 0 || (sg.x & al) || (sg.y & al) || sg.z < 0 || (sg.z & al)) return err(t, "segment alignment");
            if (sg.y != slots_end) return err(t, "segment offsets");
            if (sg.x + sg.z > n) return err(t, "segment past the vector");
            if (sg.w >= 0 && (sg.w != sg.x + sg.z || sg.w != (n & ~al) || n - sg.w < 1 || n - sg.w > al))
                return err(t, "tail columns");
            if (i > 0 && sg.x < tp.segs[seg0 + i - 1].x + tp.segs[seg0 + i - 1].z) return err(t, "segment order");
            slots_end = sg.y + sg.z + (sg.w >= 0 ? kSegAlign : 0);
            tx += sg.z;
        }
        if (tx != wtx || slots_end > kWinMax) return err(t, "window size");
        for (int k = a; k < e; ++k) {
            const int lc = tp.lcol[k];
            if (lc >= slots_end) return err(t, "local column outside the window");
            int i = nseg - 1;
            while (i > 0 && tp.segs[seg0 + i].y > lc) --i;
            const I4 sg = tp.segs[seg0 + i];
            int col = -2;
            if (lc - sg.y < sg.z) col = sg.x + (lc - sg.y);
            else if (sg.w >= 0 && lc - sg.y - sg.z < n - sg.w) col = sg.w + (lc - sg.y - sg.z);
            if (col != colidx[k]) return err(t, "local column maps to the wrong column");
        }
    }
    return std::string();
}

// SELL-32 copy of a CSR matrix (see sell.cuh): slices of 32 rows padded to
// their longest row, entries k-major within a slice; 16-bit column offsets
// from the row when all fit, else 32-bit columns.  With a slice split (the
// CTA slice ranges of the slice solve kernel), each row's entries whose
// column lies in its CTA's own rows come first (CSR order), padded to the
// slice's local width split[t], then the others (CSR order), padded to the
// slice width; padding entries are zeros at the row itself (n - 1 past n),
// which is always one of the CTA's own rows.
struct SellHost {
    std::vector<long long> ptr;
    std::vector<double> vals;
    std::vector<int16_t> cols16;
    std::vector<int32_t> cols32;
    std::vector<int32_t> split;   // local width per slice (split layout only)
    bool rel16 = true;
};

// Contiguous slice ranges for the slice solve kernel (one warp per slice): at
// most max_per_cta slices per CTA and the largest CTA cost as small as
// possible, the cost of a slice being its width (FP64 FMAs per lane in the
// SpMV) plus vec_cost (the vector work of its rows).  Binary search on the
// cost bound with a greedy fill.  Empty when the slices do not fit.
inline std::vector<int32_t> split_slices(const std::vector<long long> &ptr, int ctas, int max_per_cta,
                                         long long vec_cost) {
    const int ns = (int)ptr.size() - 1;
    if (ns < 0 || ctas < 1 || (long long)ns > (long long)ctas * max_per_cta) return {};
    std::vector<long long> cost((size_t)ns);
    long long lo = 0, hi = 0;
    for (int t = 0; t < ns; ++t) {
        cost[t] = (ptr[t + 1] - ptr[t]) / 32 + vec_cost;
        lo = std::max(lo, cost[t]);
        hi += cost[t];
    }
    auto greedy = [&](long long C, std::vector<int32_t> *cut) {
        int t = 0;
        for (int c = 0; c < ctas; ++c) {
            if (cut) (*cut)[c] = t;
            long long sum = 0;
            for (int k = 0; t < ns && k < max_per_cta && sum + cost[t] <= C; ++k) sum += cost[t++];
        }
        if (cut) (*cut)[ctas] = t;
        return t == ns;
    };
    hi = std::max(hi, lo);
    while (lo < hi) {
        const long long mid = lo + (hi - lo) / 2;
        if (greedy(mid, nullptr)) hi = mid;
        else lo = mid + 1;
    }
    std::vector<int32_t> cut((size_t)ctas + 1, 0);
    greedy(lo, &cut);
    return cut;
}

inline SellHost build_sell(int32_t n, const std::vector<int32_t> &rowptr, const std::vector<int32_t> &colidx,
                           const std::vector<double> &vals, const std::vector<int32_t> *slice_cut = nullptr) {
    SellHost S;
    const int ns = (n + 31) / 32;
    // entry order of each row: local entries first when split
    std::vector<int32_t> order(rowptr.empty() ? 0 : (size_t)rowptr[n]);
    std::vector<int32_t> nloc((size_t)n, 0);
    std::vector<int32_t> row_lo((size_t)ns, 0), row_hi((size_t)ns, n);
    if (slice_cut) {
        const int ctas = (int)slice_cut->size() - 1;
        for (int c = 0; c < ctas; ++c)
            for (int t = (*slice_cut)[c]; t < (*slice_cut)[c + 1]; ++t) {
                row_lo[t] = (*slice_cut)[c] * 32;
                row_hi[t] = std::min(n, (*slice_cut)[c + 1] * 32);
            }
    }
    for (int32_t r = 0; r < n; ++r) {
        const int t = r / 32;
        int32_t o = rowptr[r];
        for (int pass = 0; pass < (slice_cut ? 2 : 1); ++pass)
            for (int32_t k = rowptr[r]; k < rowptr[r + 1]; ++k) {
                const bool local = colidx[k] >= row_lo[t] && colidx[k] < row_hi[t];
                if (slice_cut && local != (pass == 0)) continue;
                order[o++] = k;
                if (slice_cut && local) ++nloc[r];
            }
    }
    S.ptr.assign((size_t)ns + 1, 0);
    if (slice_cut) S.split.assign((size_t)ns, 0);
    for (int t = 0; t < ns; ++t) {
        int w = 0, wl = 0, wr = 0;
        for (int r = t * 32; r < std::min(n, t * 32 + 32); ++r) {
            const int len = rowptr[r + 1] - rowptr[r];
            w = std::max(w, len);
            wl = std::max(wl, nloc[r]);
            wr = std::max(wr, len - nloc[r]);
        }
        if (slice_cut) {
            S.split[t] = wl;
            w = wl + wr;
        }
        S.ptr[t + 1] = S.ptr[t] + 32LL * w;
    }
    const size_t tot = (size_t)S.ptr[ns];
    for (int32_t r = 0; r < n && S.rel16; ++r)
        for (int32_t k = rowptr[r]; k < rowptr[r + 1]; ++k) {
            const int rel = colidx[k] - r;
            if (rel < -32768 || rel > 32767) {
                S.rel16 = false;
                break;
            }
        }
    S.vals.assign(tot, 0.0);
    if (S.rel16) S.cols16.assign(tot, 0);
    else S.cols32.assign(tot, 0);
    for (int t = 0; t < ns; ++t) {
        const int w = (int)((S.ptr[t + 1] - S.ptr[t]) / 32);
        const int wl = slice_cut ? S.split[t] : w;
        for (int l = 0; l < 32; ++l) {
            const int r = t * 32 + l;
            const int len = r < n ? rowptr[r + 1] - rowptr[r] : 0;
            const int nl = slice_cut ? (r < n ? nloc[r] : 0) : len;
            for (int k = 0; k < w; ++k) {
                const size_t idx = (size_t)S.ptr[t] + (size_t)k * 32 + l;
                int col = r < n ? r : n - 1;   // padding: value 0 at one of the CTA's own rows
                double v = 0.0;
                int e = -1;   // position in the row's entry order
                if (k < wl) {
                    if (k < nl) e = k;
                } else if (k - wl < len - nl) {
                    e = nl + (k - wl);
                }
                if (r < n && e >= 0) {
                    const int32_t src = order[rowptr[r] + e];
                    col = colidx[src];
                    v = vals[src];
                }
                S.vals[idx] = v;
                if (S.rel16) S.cols16[idx] = (int16_t)(col - r);
                else S.cols32[idx] = col;
            }
        }
    }
    return S;
}

}  // namespace gbcg
