// mfs_host.h -- multi-threaded host helpers for the set-up of a problem (ordering A's nonzeros
// into column and row order): a parallel loop and a parallel stable counting sort. Results are the
// same for any number of threads.
#pragma once

#include <sys/mman.h>

#include <algorithm>
#include <climits>
#include <atomic>
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

// Stable LSD radix sort in two passes of about half the key's bits each, on (key, item) pairs, for
// keys too many for per-thread histograms of every key. Same contract as counting_sort.
template <class Key>
void radix_sort2(int64_t n, int64_t k, Key key, const int64_t* items, int64_t* out, std::vector<int64_t>* starts) {
    const int nt = threads_for(n);
    int bits = 1;
    while ((int64_t(1) << bits) < k) ++bits;
    const int lo_bits = bits / 2;
    const int64_t nb[2] = {int64_t(1) << lo_bits, int64_t(1) << (bits - lo_bits)};
    uvec<uint32_t> k0((size_t)n), kf((size_t)n);
    uvec<int64_t> v0((size_t)n);
    std::vector<std::vector<int64_t>> cnt(nt);
    // pass: stable scatter of [0, n) by digit d of the key; src gives (key, item) of position q
    auto pass = [&](int d, auto src, uint32_t* kout, int64_t* vout) {
        const int shift = d == 0 ? 0 : lo_bits;
        const uint32_t mask = (uint32_t)(nb[d] - 1);
        for (auto& c : cnt) c.clear();
        parallel_ranges(n, nt, [&](int64_t lo, int64_t hi, int t) {
            cnt[t].assign((size_t)nb[d], 0);
            int64_t* h = cnt[t].data();
            for (int64_t q = lo; q < hi; ++q) ++h[(src(q).first >> shift) & mask];
        });
        int64_t run = 0;
        for (int64_t b = 0; b < nb[d]; ++b)
            for (int t = 0; t < nt; ++t) {
                if (cnt[t].empty()) continue;
                const int64_t c = cnt[t][b];
                cnt[t][b] = run;
                run += c;
            }
        parallel_ranges(n, nt, [&](int64_t lo, int64_t hi, int t) {
            int64_t* h = cnt[t].data();
            for (int64_t q = lo; q < hi; ++q) {
                const auto kv = src(q);
                const int64_t at = h[(kv.first >> shift) & mask]++;
                kout[at] = kv.first;
                vout[at] = kv.second;
            }
        });
    };
    pass(0, [&](int64_t q) { return std::pair<uint32_t, int64_t>((uint32_t)key(q), items ? items[q] : q); },
         k0.data(), v0.data());
    pass(1, [&](int64_t q) { return std::pair<uint32_t, int64_t>(k0[q], v0[q]); }, kf.data(), out);
    if (starts) {
        starts->assign((size_t)k + 1, n);
        int64_t* st = starts->data();
        parallel_ranges(n, nt, [&](int64_t lo, int64_t hi, int) {
            for (int64_t p = lo; p < hi; ++p)
                for (int64_t j = p ? (int64_t)kf[p - 1] + 1 : 0; j <= (int64_t)kf[p]; ++j) st[j] = p;
        });
    }
}

// Stable counting sort of the positions q in [0, n) by key(q) in [0, k): out[p] = items ? items[q] : q
// in order of (key, q). starts (nullable) receives the k+1 bucket offsets. n < 2^32. Many keys
// (more than 2^16, with several threads) go through radix_sort2 instead.
template <class Key>
void counting_sort(int64_t n, int64_t k, Key key, const int64_t* items, int64_t* out, std::vector<int64_t>* starts) {
    const int nt = threads_for(n);
    if (nt > 1 && k > (int64_t(1) << 16) && k <= (int64_t(1) << 32)) {
        radix_sort2(n, k, key, items, out, starts);
        return;
    }
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

// One order (columns or rows) of A, chunked for the warp kernels.
struct Chunks {
    std::vector<int> desc;      // 4 ints per chunk: first segment, one past last, padded offset, nnz
    std::vector<uint32_t> heads;  // 8 words per chunk: bit e set if a non-empty segment starts at item e
    std::vector<int> longs;     // chunks with more nonzeros than the limit
    int64_t padded = 0;         // length of the padded nonzero arrays
    int count() const { return (int)desc.size() / 4; }
};

// Limits of one chunk: nonzeros (a longer single segment makes a chunk of its own), segments,
// and the padding of each chunk's start in the padded nonzero arrays.
struct ChunkLimits {
    int wt, wc, pad;
};

// Greedy chunks of the segments [j0, j1) (whole units: a small Lorentz cone is one unit), with
// padded offsets and chunk numbers counted from 0.
inline void chunk_range(const std::vector<int>& ptr, int j0, int j1, const std::vector<int>* unit_end, const ChunkLimits& L,
                        Chunks& C) {
    C.desc.clear();
    C.heads.clear();
    C.longs.clear();
    C.padded = 0;
    int start = j0, cur_seg = 0;
    int64_t cur_nnz = 0;
    auto close = [&](int at) {
        const int cn = ptr[at] - ptr[start];
        if (cn > L.wt) C.longs.push_back(C.count());
        const size_t h0 = C.heads.size();
        C.heads.resize(h0 + 8, 0u);
        if (cn <= L.wt)
            for (int q = start; q < at; ++q)
                if (ptr[q + 1] > ptr[q]) {
                    const int e = ptr[q] - ptr[start];
                    C.heads[h0 + (e >> 5)] |= 1u << (e & 31);
                }
        C.desc.push_back(start);
        C.desc.push_back(at);
        C.desc.push_back((int)C.padded);
        C.desc.push_back(cn);
        C.padded += (cn + L.pad - 1) / L.pad * L.pad;
        start = at;
        cur_seg = 0;
        cur_nnz = 0;
    };
    int j = j0;
    while (j < j1) {
        const int ue = unit_end ? (*unit_end)[j] : j + 1;
        const int useg = ue - j;
        const int64_t unnz = (int64_t)ptr[ue] - ptr[j];
        if (cur_seg > 0 && (cur_nnz + unnz > L.wt || cur_seg + useg > L.wc)) close(j);
        cur_seg += useg;
        cur_nnz += unnz;
        j = ue;
        if (unnz > L.wt) close(j);
    }
    if (cur_seg > 0) close(j1);
}

// Chunks of all segments: at most L.wt nonzeros and L.wc segments each (or one segment longer than
// L.wt), greedy in segment order. The segments are cut into pieces of about 65,536 (at unit
// boundaries; the cut depends on the data only, never on the thread count) whose chunks are found
// independently, so a chunk never spans a piece boundary. `cones` lists the small Lorentz cones
// as (first, one past last) in order; unit_end[j] is the end of the unit starting at j.
struct ChunkJob {
    const std::vector<int>* ptr;
    int nseg;
    const std::vector<int>* unit_end;
    Chunks* out;
    std::vector<int> cut;
    std::vector<Chunks> part;
};

inline void plan_cuts(ChunkJob& J, const std::vector<std::pair<int, int>>& cones) {
    constexpr int PIECE = 1 << 16;
    J.cut.assign(1, 0);
    for (int j = PIECE; j < J.nseg; j += PIECE) {
        int at = j;
        if (J.unit_end) {  // not inside a small cone
            auto it = std::upper_bound(cones.begin(), cones.end(), std::make_pair(at, INT32_MAX));
            if (it != cones.begin() && std::prev(it)->second > at && std::prev(it)->first < at) at = std::prev(it)->second;
        }
        if (at > J.cut.back() && at < J.nseg) J.cut.push_back(at);
    }
    J.cut.push_back(J.nseg);
    J.part.assign(J.cut.size() - 1, Chunks());
}

// Concatenate a job's pieces: sizes and offsets first, then each piece copied by a pool thread.
struct PieceAt {
    size_t d, h, l;
    int64_t padded;
};

inline std::vector<PieceAt> size_pieces(ChunkJob& J) {
    Chunks& C = *J.out;
    std::vector<PieceAt> at(J.part.size());
    PieceAt run{0, 0, 0, 0};
    for (size_t p = 0; p < J.part.size(); ++p) {
        at[p] = run;
        run.d += J.part[p].desc.size();
        run.h += J.part[p].heads.size();
        run.l += J.part[p].longs.size();
        run.padded += J.part[p].padded;
    }
    C.desc.resize(run.d);
    C.heads.resize(run.h);
    C.longs.resize(run.l);
    C.padded = run.padded;
    return at;
}

inline void copy_piece(ChunkJob& J, const PieceAt& at, int p) {
    Chunks& C = *J.out;
    const Chunks& P = J.part[p];
    const int c0 = (int)(at.d / 4);
    for (size_t i = 0; i < P.desc.size(); i += 4) {
        C.desc[at.d + i] = P.desc[i];
        C.desc[at.d + i + 1] = P.desc[i + 1];
        C.desc[at.d + i + 2] = (int)(P.desc[i + 2] + at.padded);
        C.desc[at.d + i + 3] = P.desc[i + 3];
    }
    std::copy(P.heads.begin(), P.heads.end(), C.heads.begin() + at.h);
    for (size_t i = 0; i < P.longs.size(); ++i) C.longs[at.l + i] = P.longs[i] + c0;
}

// The chunks of several orders at once: all their pieces on one pool of threads.
inline void build_chunks(std::vector<ChunkJob>& jobs, const std::vector<std::pair<int, int>>& cones, const ChunkLimits& L) {
    std::vector<std::pair<int, int>> work;  // (job, piece)
    int64_t total = 0;
    for (int q = 0; q < (int)jobs.size(); ++q) {
        plan_cuts(jobs[q], cones);
        for (int p = 0; p + 1 < (int)jobs[q].cut.size(); ++p) work.push_back({q, p});
        total += (int64_t)(*jobs[q].ptr)[jobs[q].nseg] + jobs[q].nseg;
    }
    const int nt = std::max(1, std::min((int)work.size(), threads_for(total)));
    std::atomic<int> next{0};
    parallel_tasks(nt, [&](int) {
        for (int w = next++; w < (int)work.size(); w = next++) {
            ChunkJob& J = jobs[work[w].first];
            const int p = work[w].second;
            chunk_range(*J.ptr, J.cut[p], J.cut[p + 1], J.unit_end, L, J.part[p]);
        }
    });
    std::vector<std::vector<PieceAt>> at;
    for (ChunkJob& J : jobs) at.push_back(size_pieces(J));
    next = 0;
    parallel_tasks(nt, [&](int) {
        for (int w = next++; w < (int)work.size(); w = next++)
            copy_piece(jobs[work[w].first], at[work[w].first][work[w].second], work[w].second);
    });
}

// Argument rule of mfs_row_residuals_static, checked on the host before any device work: sizes not
// negative, n below 2^31 - 1 (as mfs_create), m within the rows that the static scratch array
// covers (max_rows), the output present, and every array that the sizes make the kernels read
// present (the CSR arrays, b and lambda when m > 0; x when n > 0).
inline bool static_resid_args_ok(int64_t m, int64_t n, int64_t max_rows, bool have_row_ptr, bool have_col_idx,
                                 bool have_val, bool have_b, bool have_x, bool have_lambda, bool have_out) {
    if (m < 0 || n < 0 || n >= INT32_MAX || m > max_rows) return false;
    if (!have_out) return false;
    if (m > 0 && !(have_row_ptr && have_col_idx && have_val && have_b && have_lambda)) return false;
    if (n > 0 && !have_x) return false;
    return true;
}

// Narrow n int64 indices to int32; returns the position of the first outside [0, lim), or n.
inline size_t narrow_indices(const int64_t* src, int32_t* dst, size_t n, int64_t lim) {
    uint64_t mx = 0;
    for (size_t i = 0; i < n; ++i) {
        const uint64_t v = (uint64_t)src[i];  // a negative index becomes huge
        mx = v > mx ? v : mx;
        dst[i] = (int32_t)src[i];
    }
    if (mx < (uint64_t)lim) return n;
    for (size_t i = 0; i < n; ++i)
        if ((uint64_t)src[i] >= (uint64_t)lim) return i;
    return n;
}

}  // namespace host
}  // namespace mfs
