// Checks mfs::host::counting_sort (counting and two-pass radix paths) against std::stable_sort on
// random keys: the permutation, the items it carries and the bucket offsets. Exit status 0 = pass.
#include <algorithm>
#include <cstdio>
#include <numeric>
#include <random>
#include <vector>

#include "mfs_host.h"

static int check(int64_t n, int64_t k, bool with_items, unsigned seed) {
    std::mt19937_64 rng(seed);
    std::vector<int64_t> key(n), items(n);
    for (int64_t q = 0; q < n; ++q) {
        key[q] = (int64_t)(rng() % (uint64_t)k);
        items[q] = (int64_t)(rng() % 1000000007ull);
    }
    std::vector<int64_t> out(n);
    std::vector<int64_t> starts;
    mfs::host::counting_sort(n, k, [&](int64_t q) { return key[q]; }, with_items ? items.data() : nullptr, out.data(),
                             &starts);
    std::vector<int64_t> ref(n);
    std::iota(ref.begin(), ref.end(), 0);
    std::stable_sort(ref.begin(), ref.end(), [&](int64_t a, int64_t b) { return key[a] < key[b]; });
    for (int64_t p = 0; p < n; ++p) {
        const int64_t want = with_items ? items[ref[p]] : ref[p];
        if (out[p] != want) {
            std::printf("n=%lld k=%lld items=%d: out[%lld] = %lld, want %lld\n", (long long)n, (long long)k,
                        (int)with_items, (long long)p, (long long)out[p], (long long)want);
            return 1;
        }
    }
    if ((int64_t)starts.size() != k + 1) {
        std::printf("n=%lld k=%lld: %zu bucket offsets\n", (long long)n, (long long)k, starts.size());
        return 1;
    }
    std::vector<int64_t> cnt(k + 1, 0);
    for (int64_t q = 0; q < n; ++q) ++cnt[key[q] + 1];
    for (int64_t j = 0; j < k; ++j) cnt[j + 1] += cnt[j];
    for (int64_t j = 0; j <= k; ++j)
        if (starts[j] != cnt[j]) {
            std::printf("n=%lld k=%lld: starts[%lld] = %lld, want %lld\n", (long long)n, (long long)k, (long long)j,
                        (long long)starts[j], (long long)cnt[j]);
            return 1;
        }
    return 0;
}

int main() {
    const int64_t sizes[][2] = {{1000, 10}, {1000, 100000}, {(1 << 20) + 7, 5}, {(1 << 20) + 7, 70000},
                                {3000000, 1000000}, {3000000, 2500000}, {2100000, 3}};
    int bad = 0;
    unsigned seed = 1;
    for (auto& s : sizes)
        for (int w = 0; w < 2; ++w) bad |= check(s[0], s[1], w == 1, seed++);
    std::printf(bad ? "FAIL\n" : "ok\n");
    return bad;
}
