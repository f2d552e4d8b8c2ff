// blink_pairs.cuh -- baseline index <-> antenna pair.
//
// Baselines are the pairs (i < j) of n antennas in lexicographic order,
// b(i, j) = i (2n - i - 1) / 2 + (j - i - 1): the cross-correlations of the
// correlation matrix's upper triangle (Sec. 4.1).  The inverse takes the row
// i from the quadratic b = i (2n - i - 1) / 2 in FP32 (good to +-1 row for
// any n < 65536) and corrects it with exact integer comparisons, so the
// result is exact.  Host and device share this code (the host side is
// checked exhaustively on the CPU).
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define BLINK_HD __host__ __device__ __forceinline__
#else
#include <cmath>
#define BLINK_HD inline
#endif

namespace blink {

BLINK_HD int64_t pair_row_start(int64_t row, int n) { return row * (2 * int64_t(n) - row - 1) / 2; }

BLINK_HD int64_t baseline_index(int i, int j, int n) { return pair_row_start(i, n) + (j - i - 1); }

BLINK_HD void baseline_pair(int64_t b, int n, int &i, int &j) {
    const int64_t t = 2 * int64_t(n) - 1;
    const float disc = float(t * t - 8 * b);
    int r = int((float(t) - sqrtf(disc > 0.f ? disc : 0.f)) * 0.5f);
    r = r < 0 ? 0 : (r > n - 2 ? n - 2 : r);
    while (r > 0 && pair_row_start(r, n) > b) --r;
    while (r < n - 2 && pair_row_start(r + 1, n) <= b) ++r;
    i = r;
    j = int(b - pair_row_start(r, n)) + r + 1;
}

}  // namespace blink

#undef BLINK_HD
