// CPU driver for the host tile planner (paper_1107_0538_gb300/csrc/plan.h):
// reads a CSR pattern (n, nnz, rowptr, colidx as raw int32 little-endian
// from a file), plans tiles and x-windows exactly as cg_create does, runs
// check_plan on the result and prints a one-line JSON summary.
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
    std::printf("{\"tiles\": %d, \"windowed\": %d, \"long\": %d, \"max_tile_nnz\": %d, "
                "\"max_segments\": %d, \"max_window_tx\": %d, \"error\": \"%s\"}\n",
                nt, tp.windowed, longs, max_nnz, maxseg, maxwin, problem.c_str());
    return problem.empty() ? 0 : 1;
}
