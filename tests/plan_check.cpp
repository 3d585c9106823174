// CPU driver for the host tile planner (paper_1107_0538_gb300/csrc/plan.h):
// reads a CSR pattern (n, nnz, rowptr, colidx as raw int32 little-endian
// from a file), plans tiles and x-windows exactly as cg_create does, runs
// check_plan on the result, builds the SELL-32 copy and checks that every
// stored entry decodes back to its CSR entry and every padded entry is a
// zero at an in-range column; prints a one-line JSON summary.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "plan.h"

int main(int argc, char **argv) {
    if (argc < 2) return 2;
    FILE *f = std::fopen(argv[1], "rb");
    if (!f) return 3;
    int32_t n = 0, nnz = 0;
    if (std::fread(&n, 4, 1, f) != 1 || std::fread(&nnz, 4, 1, f) != 1) return 4;
    std::vector<int32_t> rowptr(n + 1), colidx(nnz);
    if (std::fread(rowptr.data(), 4, n + 1, f) != (size_t)(n + 1)) return 5;
    if (nnz && std::fread(colidx.data(), 4, nnz, f) != (size_t)nnz) return 6;
    std::fclose(f);
    int max_nnz = 0;
    std::vector<int32_t> tiles = n > 0 ? gbcg::plan_tiles(n, rowptr, &max_nnz) : std::vector<int32_t>{0};
    gbcg::TilePlan tp = gbcg::plan_windows(n, rowptr, colidx, tiles);
    const std::string problem = gbcg::check_plan(n, rowptr, colidx, tiles, tp, 16);
    int longs = 0, maxseg = 0, maxwin = 0;
    const int nt = (int)tiles.size() - 1;
    for (int t = 0; t < nt; ++t) {
        const gbcg::I4 d1 = tp.desc[2 * t + 1];
        if (d1.w == gbcg::kTileLong) ++longs;
        if (d1.w == gbcg::kTileWindow) {
            maxseg = std::max(maxseg, d1.y);
            maxwin = std::max(maxwin, d1.z);
        }
    }
    // SELL-32: values are the entry numbers + 1, so each decodes uniquely
    std::vector<double> vals(nnz);
    for (int32_t k = 0; k < nnz; ++k) vals[k] = k + 1.0;
    const gbcg::SellHost sh = gbcg::build_sell(n, rowptr, colidx, vals);
    std::string sell_err;
    const int ns = (n + 31) / 32;
    if ((int)sh.ptr.size() != ns + 1 || sh.ptr[0] != 0) sell_err = "slice pointers";
    for (int t = 0; t < ns && sell_err.empty(); ++t) {
        const long long span = sh.ptr[t + 1] - sh.ptr[t];
        int w = 0;
        for (int r = t * 32; r < std::min(n, t * 32 + 32); ++r) w = std::max(w, rowptr[r + 1] - rowptr[r]);
        if (span != 32LL * w) sell_err = "slice width";
        for (int l = 0; l < 32 && sell_err.empty(); ++l) {
            const int r = t * 32 + l;
            for (int k = 0; k < w; ++k) {
                const size_t idx = (size_t)sh.ptr[t] + (size_t)k * 32 + l;
                const int col = sh.rel16 ? r + sh.cols16[idx] : sh.cols32[idx];
                const bool real = r < n && k < rowptr[r + 1] - rowptr[r];
                if (col < 0 || col >= n) { sell_err = "column out of range"; break; }
                if (real && (col != colidx[rowptr[r] + k] || sh.vals[idx] != vals[rowptr[r] + k])) {
                    sell_err = "entry does not decode";
                    break;
                }
                if (!real && sh.vals[idx] != 0.0) { sell_err = "nonzero padding"; break; }
            }
        }
    }
    // slice split of the slice solve kernel (152 CTAs, 31 slices each at most)
    const int ctas = 152, per = 31;
    const std::vector<int32_t> cut = gbcg::split_slices(sh.ptr, ctas, per, 8);
    long long slice_cost = -1, slice_bound = 0, total = 0;
    if (!cut.empty()) {
        if ((int)cut.size() != ctas + 1 || cut[0] != 0 || cut[ctas] != ns) sell_err = "slice split bounds";
        slice_cost = 0;
        for (int c = 0; c < ctas && sell_err.empty(); ++c) {
            if (cut[c + 1] < cut[c] || cut[c + 1] - cut[c] > per) sell_err = "slice split range";
            long long cc = 0;
            for (int t = cut[c]; t < cut[c + 1]; ++t) cc += (sh.ptr[t + 1] - sh.ptr[t]) / 32 + 8;
            slice_cost = std::max(slice_cost, cc);
        }
        for (int t = 0; t < ns; ++t) {
            const long long ct = (sh.ptr[t + 1] - sh.ptr[t]) / 32 + 8;
            total += ct;
            slice_bound = std::max(slice_bound, ct);
        }
        slice_bound = std::max(slice_bound, (total + ctas - 1) / ctas);
        // the split layout: every entry of a slice's local block (padding too)
        // lies in the CTA's own rows; each row keeps exactly its CSR entries
        const gbcg::SellHost sp = gbcg::build_sell(n, rowptr, colidx, vals, &cut);
        if ((int)sp.ptr.size() != ns + 1 || (int)sp.split.size() != ns || sp.rel16 != sh.rel16)
            sell_err = "split layout sizes";
        for (int c = 0; c < ctas && sell_err.empty(); ++c) {
            const int r0 = cut[c] * 32, r1 = std::min(n, cut[c + 1] * 32);
            for (int t = cut[c]; t < cut[c + 1] && sell_err.empty(); ++t) {
                const int w = (int)((sp.ptr[t + 1] - sp.ptr[t]) / 32);
                if (sp.split[t] < 0 || sp.split[t] > w) { sell_err = "split width"; break; }
                for (int l = 0; l < 32 && sell_err.empty(); ++l) {
                    const int r = t * 32 + l;
                    std::vector<long long> seen;
                    for (int k = 0; k < w; ++k) {
                        const size_t idx = (size_t)sp.ptr[t] + (size_t)k * 32 + l;
                        const int col = sp.rel16 ? r + sp.cols16[idx] : sp.cols32[idx];
                        if (col < 0 || col >= n) { sell_err = "split column out of range"; break; }
                        if (k < sp.split[t] && (col < r0 || col >= r1)) { sell_err = "remote column in local block"; break; }
                        const double v = sp.vals[idx];
                        if (v == 0.0) continue;
                        const long long e = (long long)v - 1;
                        if (r >= n || e < rowptr[r] || e >= rowptr[r + 1] || colidx[e] != col) {
                            sell_err = "split entry does not decode";
                            break;
                        }
                        seen.push_back(e);
                    }
                    if (!sell_err.empty()) break;
                    std::sort(seen.begin(), seen.end());
                    const long long len = r < n ? rowptr[r + 1] - rowptr[r] : 0;
                    bool ok = (long long)seen.size() == len;
                    for (long long i = 0; ok && i < len; ++i) ok = seen[i] == rowptr[r] + i;
                    if (!ok) sell_err = "split row entries";
                }
            }
        }
    } else if (ns <= ctas * per) {
        sell_err = "slice split missing";
    }
    bool fits = true;
    for (int32_t r = 0; r < n; ++r)
        for (int32_t k = rowptr[r]; k < rowptr[r + 1]; ++k)
            if (colidx[k] - r < -32768 || colidx[k] - r > 32767) fits = false;
    if (sell_err.empty() && fits != sh.rel16) sell_err = "wrong column width";
    std::printf("{\"tiles\": %d, \"windowed\": %d, \"long\": %d, \"max_tile_nnz\": %d, "
                "\"max_segments\": %d, \"max_window_tx\": %d, \"sell_entries\": %lld, \"sell_rel16\": %d, "
                "\"slice_cost\": %lld, \"slice_bound\": %lld, \"error\": \"%s%s\"}\n",
                nt, tp.windowed, longs, max_nnz, maxseg, maxwin, (long long)sh.ptr.back(), (int)sh.rel16,
                slice_cost, slice_bound, problem.c_str(), sell_err.c_str());
    return problem.empty() && sell_err.empty() ? 0 : 1;
}
