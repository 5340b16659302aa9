// Checks mfs::host::build_chunks (the chunk plan of both orders of A) against the rules it must
// follow, on random segment lengths with empty, short and long segments and small cones: the
// chunks tile the segments in order; a chunk holds at most wt nonzeros and wc segments, or is one
// unit longer than wt and is then listed as long; no chunk boundary falls inside a small cone;
// padded offsets are the running sums of the nonzero counts rounded up to pad; the head bits mark
// exactly the local positions where a non-empty segment starts; every chunk that does not end a
// piece could not take the next unit (greedy); pieces break at multiples of 65,536 segments,
// moved past a cone that straddles them. Exit status 0 = pass.
#include <algorithm>
#include <cstdio>
#include <random>
#include <utility>
#include <vector>

#include "mfs_host.h"

using mfs::host::ChunkJob;
using mfs::host::ChunkLimits;
using mfs::host::Chunks;

static int fail(const char* what, int c) {
    std::printf("FAIL: %s (chunk %d)\n", what, c);
    return 1;
}

static int check(const std::vector<int>& ptr, const std::vector<int>* unit_end,
                 const std::vector<std::pair<int, int>>& cones, const ChunkLimits& L, const Chunks& C) {
    const int nseg = (int)ptr.size() - 1;
    std::vector<char> inside(nseg + 1, 0);  // a boundary at j would split a cone
    for (const auto& q : cones)
        for (int j = q.first + 1; j < q.second; ++j) inside[j] = 1;
    // piece boundaries: every multiple of 65,536, moved to the end of a cone that straddles it
    std::vector<char> cut(nseg + 1, 0);
    for (int j = 65536; j < nseg; j += 65536) {
        int at = j;
        for (const auto& q : cones)
            if (q.first < j && j < q.second) at = q.second;
        if (at < nseg) cut[at] = 1;
    }
    int64_t padded = 0;
    int at = 0;
    size_t nlong = 0;
    for (int c = 0; c < C.count(); ++c) {
        const int s0 = C.desc[4 * c], s1 = C.desc[4 * c + 1], off = C.desc[4 * c + 2], cn = C.desc[4 * c + 3];
        if (s0 != at || s1 <= s0) return fail("chunks do not tile the segments in order", c);
        if (inside[s0] || inside[s1]) return fail("boundary inside a small cone", c);
        if (cn != ptr[s1] - ptr[s0]) return fail("nonzero count", c);
        if (off != padded) return fail("padded offset", c);
        padded += (cn + L.pad - 1) / L.pad * L.pad;
        if (s1 - s0 > L.wc) return fail("too many segments", c);
        const bool single_unit = unit_end ? (*unit_end)[s0] == s1 : s1 == s0 + 1;
        const bool is_long = cn > L.wt;
        if (is_long && !single_unit) return fail("more than wt nonzeros in several units", c);
        if (is_long) {
            if (nlong >= C.longs.size() || C.longs[nlong] != c) return fail("long chunk not listed in order", c);
            ++nlong;
        } else {
            for (int e = 0; e < 32 * 8 && e < L.wt; ++e) {
                bool head = false;
                for (int q = s0; q < s1; ++q)
                    if (ptr[q + 1] > ptr[q] && ptr[q] - ptr[s0] == e) head = true;
                const bool bit = (C.heads[8 * (size_t)c + (e >> 5)] >> (e & 31)) & 1u;
                if (bit != head) return fail("head bits", c);
            }
        }
        // greedy: unless a piece ends here, the next unit did not fit
        if (!cut[s1] && !is_long && s1 < nseg) {
            const int ue = unit_end ? (*unit_end)[s1] : s1 + 1;
            const int64_t unnz = ptr[ue] - ptr[s1];
            const bool fits = unnz <= L.wt && cn + unnz <= L.wt && (s1 - s0) + (ue - s1) <= L.wc;
            if (fits) return fail("not greedy: the next unit would have fit", c);
        }
        at = s1;
    }
    if (at != nseg) return fail("chunks end before the last segment", C.count());
    if (nlong != C.longs.size()) return fail("extra long chunks listed", C.count());
    if (padded != C.padded) return fail("padded length", C.count());
    return 0;
}

int main() {
    const ChunkLimits L{256, 64, 8};
    std::mt19937 rng(7);
    int bad = 0;
    for (int trial = 0; trial < 6; ++trial) {
        const int n = trial == 0 ? 0 : trial == 1 ? 1000 : trial == 2 ? 70000 : 300000 + 12345 * trial;
        const int m = trial == 0 ? 0 : n / 3 + 7;
        std::vector<int> ptr(n + 1, 0), rptr(m + 1, 0);
        std::geometric_distribution<int> deg(trial == 3 ? 0.5 : 0.12);
        for (int j = 0; j < n; ++j) {
            int d = (trial == 4) ? 0 : deg(rng);               // trial 4: all segments empty
            if (trial >= 3 && rng() % 5000 == 0) d = 300 + (int)(rng() % 2000);  // long segments
            ptr[j + 1] = ptr[j] + d;
        }
        std::geometric_distribution<int> rdeg(0.05);
        for (int i = 0; i < m; ++i) rptr[i + 1] = rptr[i] + rdeg(rng);
        // small cones (at most 64 columns and 256 nonzeros), some straddling a piece boundary
        std::vector<int> ue(n);
        for (int j = 0; j < n; ++j) ue[j] = j + 1;
        std::vector<std::pair<int, int>> cones;
        for (int s = 40; s + 70 < n; s += 997 + (int)(rng() % 5000)) {
            const int sz = 2 + (int)(rng() % 40);
            if (ptr[s + sz] - ptr[s] > L.wt) continue;
            if (!cones.empty() && cones.back().second > s) continue;
            cones.push_back({s, s + sz});
            ue[s] = s + sz;
        }
        for (int b = 65536; b + 64 < n; b += 65536) {  // one cone across each piece boundary
            const int s = b - 5, sz = 20;
            bool clash = false;
            for (const auto& q : cones)
                if (q.second > s - 1 && q.first < s + sz + 1) clash = true;
            if (clash || ptr[s + sz] - ptr[s] > L.wt) continue;
            cones.push_back({s, s + sz});
            ue[s] = s + sz;
        }
        std::sort(cones.begin(), cones.end());
        Chunks C, R;
        std::vector<ChunkJob> jobs(2);
        jobs[0].ptr = &ptr;
        jobs[0].nseg = n;
        jobs[0].unit_end = &ue;
        jobs[0].out = &C;
        jobs[1].ptr = &rptr;
        jobs[1].nseg = m;
        jobs[1].unit_end = nullptr;
        jobs[1].out = &R;
        mfs::host::build_chunks(jobs, cones, L);
        if (check(ptr, &ue, cones, L, C)) {
            std::printf("  columns, trial %d (n = %d)\n", trial, n);
            bad = 1;
        }
        if (check(rptr, nullptr, {}, L, R)) {
            std::printf("  rows, trial %d (m = %d)\n", trial, m);
            bad = 1;
        }
        // the same plan when built again (no dependence on thread timing)
        Chunks C2, R2;
        jobs[0].out = &C2;
        jobs[1].out = &R2;
        mfs::host::build_chunks(jobs, cones, L);
        if (C2.desc != C.desc || C2.heads != C.heads || C2.longs != C.longs || R2.desc != R.desc) {
            std::printf("FAIL: plan differs between two runs, trial %d\n", trial);
            bad = 1;
        }
    }
    if (!bad) std::printf("ok\n");
    return bad;
}
