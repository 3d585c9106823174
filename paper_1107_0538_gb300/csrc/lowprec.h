// Host-side construction of the low-precision inner matrix used by the
// mixed-precision solve (plain C++, no CUDA calls).
//
// Every off-diagonal value is rounded to nearest, ties to even, into FP32 or
// BF16.  Rounding alone would move each row sum by up to half an ulp per
// entry; for a stiffness matrix (rows summing to zero) plus a small mass
// shift that destroys the smallest eigenvalues.  So the inner diagonal is
// kept apart, in FP32, as the row sum of A minus the row sum of the rounded
// off-diagonals (both summed in FP64 in storage order): the inner matrix
// keeps A's row sums up to one FP32 rounding.  For a symmetric matrix with
// non-positive off-diagonals this makes it a relative perturbation of each
// coupling, so its spectrum stays within a factor 1 +- eps of A's.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace gbcg {

// Round a double to the nearest BF16 (ties to even) with one rounding, from
// the bits: keep 8 significant bits (fewer below 2^-126, where BF16 is
// subnormal), round the dropped bits, overflow to infinity.
inline uint16_t bf16_bits_rne(double v) {
    uint64_t u;
    std::memcpy(&u, &v, 8);
    const uint16_t sign = (uint16_t)((u >> 63) << 15);
    const int exp = (int)((u >> 52) & 0x7ff);
    const uint64_t frac = u & ((1ull << 52) - 1);
    if (exp == 0x7ff) return (uint16_t)(sign | (frac ? 0x7fc0 : 0x7f80));  // NaN / infinity
    if (exp == 0) return sign;  // double subnormals are far below the smallest BF16
    const int E = exp - 1023;                 // v = 1.frac * 2^E
    const uint64_t sig = (1ull << 52) | frac; // 53 significant bits
    int drop = 45;                            // keep 8 of them
    if (E < -126) drop += -126 - E;           // BF16 subnormal: fewer bits
    if (drop > 54) return sign;               // below half the smallest subnormal
    uint64_t kept = sig >> drop;
    const uint64_t rem = sig & ((1ull << drop) - 1), half = 1ull << (drop - 1);
    if (rem > half || (rem == half && (kept & 1))) ++kept;
    // value = kept * 2^(E - 52 + drop), exactly representable in BF16 and FP32
    const double r = std::ldexp((double)kept, E - 52 + drop);
    if (r >= 0x1p128) return (uint16_t)(sign | 0x7f80);
    float f = (float)r;  // exact
    uint32_t fb;
    std::memcpy(&fb, &f, 4);
    return (uint16_t)(sign | (uint16_t)(fb >> 16));
}

inline double bf16_to_double(uint16_t b) {
    const uint32_t fb = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &fb, 4);
    return (double)f;
}

struct InnerMatrix {
    std::vector<float> vals32;     // FP32 values (diagonal slots 0), when fp32
    std::vector<uint16_t> vals16;  // BF16 values (diagonal slots 0), when bf16
    std::vector<float> diag;       // compensated FP32 diagonal per row (0 when absent)
};

// fmt 1 = FP32 off-diagonals, 2 = BF16 off-diagonals.
inline InnerMatrix build_inner(int32_t n, const std::vector<int32_t> &rowptr,
                               const std::vector<int32_t> &colidx, const std::vector<double> &vals,
                               int fmt) {
    InnerMatrix M;
    const size_t nnz = vals.size();
    if (fmt == 1) M.vals32.assign(nnz, 0.0f);
    else M.vals16.assign(nnz, 0);
    M.diag.assign((size_t)n, 0.0f);
    for (int32_t i = 0; i < n; ++i) {
        double rowsum = 0.0, offsum = 0.0;
        bool has_diag = false;
        for (int32_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            rowsum += vals[k];
            if (colidx[k] == i) {
                has_diag = true;
                continue;  // stored as 0 in the value array
            }
            double lo;
            if (fmt == 1) {
                M.vals32[k] = (float)vals[k];  // IEEE conversion: nearest, ties to even
                lo = (double)M.vals32[k];
            } else {
                M.vals16[k] = bf16_bits_rne(vals[k]);
                lo = bf16_to_double(M.vals16[k]);
            }
            offsum += lo;
        }
        if (has_diag) M.diag[i] = (float)(rowsum - offsum);
    }
    return M;
}

}  // namespace gbcg
