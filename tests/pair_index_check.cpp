// Exhaustive host check of blink::baseline_pair against the lexicographic
// enumeration of the pairs (i < j); prints "ok <count>" or the first mismatch.
#include <cstdio>
#include <cstdlib>

#include "blink_pairs.cuh"

static int check_all(int n, long long &count) {
    long long b = 0;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j, ++b) {
            int pi, pj;
            blink::baseline_pair(b, n, pi, pj);
            if (pi != i || pj != j || blink::baseline_index(i, j, n) != b) {
                std::printf("mismatch n=%d b=%lld: (%d,%d) vs (%d,%d)\n", n, b, pi, pj, i, j);
                return 1;
            }
            ++count;
        }
    return 0;
}

// Large arrays: every row's first and last baseline and its neighbours.
static int check_rows(int n, long long &count) {
    for (int i = 0; i < n - 1; ++i) {
        const long long s = blink::pair_row_start(i, n), e = s + (n - i - 1) - 1;
        const long long probes[4] = {s, s + 1 < e ? s + 1 : s, e - 1 > s ? e - 1 : e, e};
        for (long long b : probes) {
            int pi, pj;
            blink::baseline_pair(b, n, pi, pj);
            if (pi != i || pj != int(b - s) + i + 1) {
                std::printf("mismatch n=%d b=%lld: (%d,%d) expected row %d\n", n, b, pi, pj, i);
                return 1;
            }
            ++count;
        }
    }
    return 0;
}

int main() {
    long long count = 0;
    for (int n = 2; n <= 700; ++n)
        if (check_all(n, count)) return 1;
    const int big[] = {1024, 2048, 4095, 4096, 8192, 16383, 32768, 65535};
    for (int n : big)
        if (check_rows(n, count)) return 1;
    if (check_all(4096, count)) return 1;
    std::printf("ok %lld\n", count);
    return 0;
}
