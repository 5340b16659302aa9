// Checks mfs::host::narrow_indices (int64 COO indices narrowed to int32 for the upload, each
// checked against [0, lim) first): every valid index comes through unchanged, and the reported
// position is the first index that is negative, at or above the limit, or beyond int32 (including
// values that would wrap to a valid int32). Exit status 0 = pass.
#include <cstdio>
#include <random>
#include <vector>

#include "mfs_host.h"

int main() {
    std::mt19937_64 rng(3);
    int bad = 0;
    const int64_t lim = 1000003;
    const int64_t wild[] = {-1, lim, lim + 7, (int64_t(1) << 32) + 5, -(int64_t(1) << 32) + 3,
                            (int64_t(1) << 31), INT64_MIN, INT64_MAX};
    for (int trial = 0; trial < 200; ++trial) {
        const size_t n = trial == 0 ? 0 : 1 + rng() % 5000;
        std::vector<int64_t> src(n);
        for (auto& v : src) v = (int64_t)(rng() % (uint64_t)lim);
        size_t first = n;
        if (trial % 3 != 0 && n > 0) {  // plant one to three bad indices
            const int k = 1 + (int)(rng() % 3);
            for (int q = 0; q < k; ++q) {
                const size_t at = rng() % n;
                src[at] = wild[rng() % (sizeof wild / sizeof wild[0])];
                first = std::min(first, at);
            }
        }
        std::vector<int32_t> dst(n, -7);
        const size_t got = mfs::host::narrow_indices(src.data(), dst.data(), n, lim);
        if (got != first) {
            std::printf("FAIL: trial %d: first bad at %zu, reported %zu\n", trial, first, got);
            bad = 1;
        }
        for (size_t i = 0; i < n; ++i)
            if (src[i] >= 0 && src[i] < lim && dst[i] != (int32_t)src[i]) {
                std::printf("FAIL: trial %d: index %zu narrowed to %d, want %lld\n", trial, i, dst[i], (long long)src[i]);
                bad = 1;
                break;
            }
    }
    if (!bad) std::printf("ok\n");
    return bad;
}
