// mfs_host.h -- multi-threaded host helpers for the set-up of a problem (ordering A's nonzeros
// into column and row order): a parallel loop and a parallel stable counting sort. Results are the
// same for any number of threads.
#pragma once

#include <sys/mman.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <memory>
#include <new>
#include <thread>
#include <utility>
#include <vector>

namespace mfs {
namespace host {

// Allocator for the large set-up arrays: resize() leaves new elements uninitialised (the threads
// that fill them are the first to write), and blocks of 4 MiB or more are 2 MiB aligned and
// advised to use huge pages, so that the first writes fault in 2 MiB at a time.
template <class T>
struct uninit_alloc : std::allocator<T> {
    template <class U>
    struct rebind {
        using other = uninit_alloc<U>;
    };
    static constexpr size_t kHuge = size_t(2) << 20;
    uninit_alloc() = default;
    template <class U>
    uninit_alloc(const uninit_alloc<U>&) noexcept {}
    T* allocate(size_t n) {
        const size_t bytes = n * sizeof(T);
        if (bytes < 2 * kHuge) return std::allocator<T>::allocate(n);
        const size_t len = (bytes + kHuge - 1) / kHuge * kHuge;
        void* p = std::aligned_alloc(kHuge, len);
        if (!p) throw std::bad_alloc();
        madvise(p, len, MADV_HUGEPAGE);
        return static_cast<T*>(p);
    }
    void deallocate(T* p, size_t n) noexcept {
        if (n * sizeof(T) < 2 * kHuge)
            std::allocator<T>::deallocate(p, n);
        else
            std::free(p);
    }
    template <class U>
    void construct(U*) noexcept {}
    template <class U, class... A>
    void construct(U* p, A&&... a) {
        ::new ((void*)p) U(std::forward<A>(a)...);
    }
};
template <class T>
using uvec = std::vector<T, uninit_alloc<T>>;

// Threads for a pass over `work` items: one below 2^20 items, else the hardware's (at most 32).
inline int threads_for(int64_t work) {
    if (work < (int64_t(1) << 20)) return 1;
    const unsigned h = std::thread::hardware_concurrency();
    return (int)std::max(1u, std::min(h ? h : 1u, 32u));
}

// f(lo, hi, t) on nt contiguous ranges of [0, n), one thread each.
template <class F>
void parallel_ranges(int64_t n, int nt, F f) {
    if (nt <= 1 || n < 2 * nt) {
        f(int64_t(0), n, 0);
        return;
    }
    std::vector<std::thread> pool;
    pool.reserve(nt - 1);
    for (int t = 1; t < nt; ++t) pool.emplace_back([&, t] { f(n * t / nt, n * (t + 1) / nt, t); });
    f(0, n / nt, 0);
    for (auto& th : pool) th.join();
}

// f(t) for t in [0, nt), each on its own thread.
template <class F>
void parallel_tasks(int nt, F f) {
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; ++t) pool.emplace_back([&, t] { f(t); });
    if (nt > 0) f(0);
    for (auto& th : pool) th.join();
}

// Stable counting sort of the positions q in [0, n) by key(q) in [0, k): out[p] = items ? items[q] : q
// in order of (key, q). starts (nullable) receives the k+1 bucket offsets. n < 2^32.
template <class Key>
void counting_sort(int64_t n, int64_t k, Key key, const int64_t* items, int64_t* out, std::vector<int64_t>* starts) {
    const int nt = threads_for(n);
    // cnt[t][b]: entries of bucket b in thread t's range; then, in place, where thread t writes its
    // first entry of bucket b: all entries of smaller buckets plus those of b in threads < t
    std::vector<std::vector<uint32_t>> cnt(nt, std::vector<uint32_t>((size_t)k, 0u));
    parallel_ranges(n, nt, [&](int64_t lo, int64_t hi, int t) {
        uint32_t* h = cnt[t].data();
        for (int64_t q = lo; q < hi; ++q) ++h[key(q)];
    });
    std::vector<int64_t> total((size_t)k + 1, 0);
    parallel_ranges(k, nt, [&](int64_t lo, int64_t hi, int) {
        for (int64_t b = lo; b < hi; ++b) {
            int64_t s = 0;
            for (int t = 0; t < nt; ++t) s += cnt[t][b];
            total[b + 1] = s;
        }
    });
    for (int64_t b = 0; b < k; ++b) total[b + 1] += total[b];
    parallel_ranges(k, nt, [&](int64_t lo, int64_t hi, int) {
        for (int64_t b = lo; b < hi; ++b) {
            int64_t run = total[b];
            for (int t = 0; t < nt; ++t) {
                const uint32_t c = cnt[t][b];
                cnt[t][b] = (uint32_t)run;
                run += c;
            }
        }
    });
    parallel_ranges(n, nt, [&](int64_t lo, int64_t hi, int t) {
        uint32_t* p = cnt[t].data();
        for (int64_t q = lo; q < hi; ++q) out[p[key(q)]++] = items ? items[q] : q;
    });
    if (starts) starts->assign(total.begin(), total.end());
}

}  // namespace host
}  // namespace mfs
