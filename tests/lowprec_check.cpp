// CPU driver for the library's inner-matrix construction (csrc/lowprec.h):
// reads a CSR matrix (n, nnz, rowptr, colidx as int32, vals as f64) and a
// format (1 = FP32, 2 = BF16), builds the inner matrix as cg_create does and
// writes it back in the oracle's layout (doubles, the compensated diagonal in
// the row's first diagonal slot, 0 in further diagonal slots).
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "lowprec.h"

int main(int argc, char **argv) {
    if (argc < 4) return 2;
    FILE *f = std::fopen(argv[1], "rb");
    if (!f) return 3;
    int32_t n = 0, nnz = 0;
    if (std::fread(&n, 4, 1, f) != 1 || std::fread(&nnz, 4, 1, f) != 1) return 4;
    std::vector<int32_t> rowptr(n + 1), colidx(nnz);
    std::vector<double> vals(nnz);
    if (std::fread(rowptr.data(), 4, n + 1, f) != (size_t)(n + 1)) return 5;
    if (nnz && std::fread(colidx.data(), 4, nnz, f) != (size_t)nnz) return 6;
    if (nnz && std::fread(vals.data(), 8, nnz, f) != (size_t)nnz) return 7;
    std::fclose(f);
    const int fmt = std::atoi(argv[2]);
    gbcg::InnerMatrix M = gbcg::build_inner(n, rowptr, colidx, vals, fmt);
    std::vector<double> out(nnz);
    for (int32_t i = 0; i < n; ++i) {
        bool first = true;
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            if (colidx[k] == i) {
                out[k] = first ? (double)M.diag[i] : 0.0;
                first = false;
            } else {
                out[k] = fmt == 1 ? (double)M.vals32[k] : gbcg::bf16_to_double(M.vals16[k]);
            }
        }
    }
    FILE *g = std::fopen(argv[3], "wb");
    if (!g) return 8;
    std::fwrite(out.data(), 8, nnz, g);
    std::fclose(g);
    return 0;
}
