// mfs_setup.cuh -- set-up of A on the GPU (Algorithm 1, steps 1-3: the nonzeros in column order,
// the U V decomposition's orders and the padded chunk layouts) for COO input that arrives already in
// column order (rows ascending within a column, duplicates next to each other). The host then only
// chunks the column and row pointer arrays.
//
// From the uploaded COO (int64 indices, FP64 values): a check of every entry (first index out of
// range, first non-finite value, order); runs of equal (column, row) summed and runs summing to
// zero dropped (a device-wide scan gives the compacted positions); column pointers; the row order
// by a count, a scan and a scatter, each row then sorted by column, so that it equals the stable
// order the host builds; finally the nonzeros are copied into the chunks' padded slots.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mfs {
namespace setup {

constexpr int NT = 256;
constexpr int IT = 8;                  // items per thread of a scan block
constexpr int SPAN = NT * IT;          // items per scan block

// ------------------------------------------------------------------------------------ scan
// Exclusive scan of n ints in three launches: per-block scans with the block totals, a scan of the
// totals by one block, the totals added back. total (nullable) receives the sum of all n.
__global__ void __launch_bounds__(NT) k_scan_local(const int* __restrict__ in, int* __restrict__ out,
                                                   int* __restrict__ blk, long long n) {
    __shared__ int sw[NT / 32];
    const long long base = (long long)blockIdx.x * SPAN + (long long)threadIdx.x * IT;
    int v[IT];
    int s = 0;
#pragma unroll
    for (int q = 0; q < IT; ++q) {
        v[q] = base + q < n ? in[base + q] : 0;
        s += v[q];
    }
    // inclusive scan of the thread sums over the block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int o = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += o;
    }
    if (lane == 31) sw[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < NT / 32 ? sw[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += o;
        }
        if (lane < NT / 32) sw[lane] = w;
    }
    __syncthreads();
    int run = x - s + (warp > 0 ? sw[warp - 1] : 0);  // exclusive prefix of this thread
#pragma unroll
    for (int q = 0; q < IT; ++q) {
        if (base + q < n) out[base + q] = run;
        run += v[q];
    }
    if (threadIdx.x == NT - 1) blk[blockIdx.x] = run;
}

__global__ void __launch_bounds__(1024) k_scan_blocks(int* __restrict__ blk, int nb, int* __restrict__ total) {
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    __shared__ int sw[32];
    for (int b0 = 0; b0 < nb; b0 += 1024) {
        const int i = b0 + threadIdx.x;
        const int s = i < nb ? blk[i] : 0;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        int x = s;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += o;
        }
        if (lane == 31) sw[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int w = sw[lane];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int o = __shfl_up_sync(0xffffffffu, w, d);
                if (lane >= d) w += o;
            }
            sw[lane] = w;
        }
        __syncthreads();
        const int incl = x + (warp > 0 ? sw[warp - 1] : 0);
        if (i < nb) blk[i] = carry + incl - s;
        __syncthreads();
        if (threadIdx.x == 1023) carry += incl;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void __launch_bounds__(NT) k_scan_add(int* __restrict__ out, const int* __restrict__ blk, long long n) {
    const long long base = (long long)blockIdx.x * SPAN + (long long)threadIdx.x * IT;
    const int add = blk[blockIdx.x];
#pragma unroll
    for (int q = 0; q < IT; ++q)
        if (base + q < n) out[base + q] += add;
}

// ------------------------------------------------------------------------------------ COO input
// First entry with an index out of range, first non-finite value (atomic minima; nnz if none), and
// whether some entry comes before its predecessor in (column, row) order. The indices arrive as
// int32, narrowed on the host after their own range check there.
__global__ void k_check(const int* __restrict__ row, const int* __restrict__ col,
                        const double* __restrict__ val, long long nnz, long long m, long long n,
                        unsigned long long* bad_idx, unsigned long long* bad_val, int* unsorted) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nnz; q += (long long)gridDim.x * blockDim.x) {
        const long long r = row[q], c = col[q];
        if (r < 0 || r >= m || c < 0 || c >= n) atomicMin(bad_idx, (unsigned long long)q);
        if (!isfinite(val[q])) atomicMin(bad_val, (unsigned long long)q);
        if (q + 1 < nnz) {
            const long long c1 = col[q + 1], r1 = row[q + 1];
            if (c > c1 || (c == c1 && r > r1)) *unsorted = 1;
        }
    }
}

// COO indices that already live on the device (mfs_create_device): int64 narrowed to int32, an
// index outside [0, lim) becoming -1 so that k_check reports its position.
__global__ void k_narrow_dev(const long long* __restrict__ src, long long nnz, long long lim, int* __restrict__ dst) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nnz; q += (long long)gridDim.x * blockDim.x) {
        const long long v = src[q];
        dst[q] = (v >= 0 && v < lim) ? (int)v : -1;
    }
}

// flag = 1 if some element of p[0 .. n) is NaN or infinite
__global__ void k_nonfinite(const double* __restrict__ p, long long n, int* __restrict__ flag) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        if (!isfinite(p[q])) *flag = 1;
}

// In column order (duplicates allowed): keep[q] = 1 where a run of equal (column, row) starts and
// its values sum to a nonzero, sum[q] = that sum (in entry order).
__global__ void k_runs(const int* __restrict__ row, const int* __restrict__ col,
                       const double* __restrict__ val, long long nnz, int* __restrict__ keep, double* __restrict__ sum) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nnz; q += (long long)gridDim.x * blockDim.x) {
        const long long r = row[q], c = col[q];
        const bool head = q == 0 || row[q - 1] != r || col[q - 1] != c;
        int k = 0;
        if (head) {
            double s = val[q];
            for (long long e = q + 1; e < nnz && row[e] == r && col[e] == c; ++e) s += val[e];
            sum[q] = s;
            k = s != 0.0;
        }
        keep[q] = k;
    }
}

__global__ void k_compact(const int* __restrict__ row, const int* __restrict__ col,
                          const int* __restrict__ keep, const int* __restrict__ pos, const double* __restrict__ sum,
                          long long nnz, int* __restrict__ crow, int* __restrict__ ccol, double* __restrict__ cval) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nnz; q += (long long)gridDim.x * blockDim.x)
        if (keep[q]) {
            const int p = pos[q];
            crow[p] = (int)row[q];
            ccol[p] = (int)col[q];
            cval[p] = sum[q];
        }
}

// ptr[j] = first position p with seg[p] >= j, for j in [0, nseg], from sorted seg[0 .. o).
__global__ void k_seg_ptr(const int* __restrict__ seg, long long o, int nseg, int* __restrict__ ptr) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < o; p += (long long)gridDim.x * blockDim.x) {
        const int lo = p == 0 ? 0 : seg[p - 1] + 1;
        for (int j = lo; j <= seg[p]; ++j) ptr[j] = (int)p;
        if (p == o - 1)
            for (int j = seg[p] + 1; j <= nseg; ++j) ptr[j] = (int)o;
    }
}

__global__ void k_count(const int* __restrict__ key, long long o, int* __restrict__ cnt) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < o; p += (long long)gridDim.x * blockDim.x)
        atomicAdd(cnt + key[p], 1);
}

// Row order: each column-order entry into a free slot of its row (the order inside a row is then
// fixed by k_sort_rows).
__global__ void k_scatter_rows(const int* __restrict__ crow, const int* __restrict__ ccol,
                               const double* __restrict__ cval, long long o, const int* __restrict__ row_ptr,
                               int* __restrict__ fill, int* __restrict__ rcol, double* __restrict__ rval) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < o; p += (long long)gridDim.x * blockDim.x) {
        const int r = crow[p];
        const int at = row_ptr[r] + atomicAdd(fill + r, 1);
        rcol[at] = ccol[p];
        rval[at] = cval[p];
    }
}

// Each row's entries by ascending column (columns are distinct within a row): insertion sort for
// short rows, Shell sort (Ciura's gaps) for long ones; one thread per row.
__global__ void k_sort_rows(const int* __restrict__ row_ptr, int m, int* __restrict__ rcol, double* __restrict__ rval) {
    const int gaps[8] = {701, 301, 132, 57, 23, 10, 4, 1};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const int a = row_ptr[i], e = row_ptr[i + 1], len = e - a;
        for (int gi = 0; gi < 8; ++gi) {
            const int gap = gaps[gi];
            if (gap >= len) continue;
            for (int q = a + gap; q < e; ++q) {
                const int c = rcol[q];
                const double v = rval[q];
                int w = q;
                while (w - gap >= a && rcol[w - gap] > c) {
                    rcol[w] = rcol[w - gap];
                    rval[w] = rval[w - gap];
                    w -= gap;
                }
                rcol[w] = c;
                rval[w] = v;
            }
        }
    }
}

// ------------------------------------------------------------------------------------ padding
// Chunk c's nonzeros (segments desc.x .. desc.y-1, ptr giving their range in the unpadded order)
// into its padded slots from desc.z; one warp per chunk. The other slots are zeroed beforehand.
template <typename T>
__global__ void k_pad(const int4* __restrict__ desc, int nchunks, const int* __restrict__ ptr,
                      const int* __restrict__ idx, const double* __restrict__ val, int* __restrict__ pidx,
                      T* __restrict__ pval) {
    const int lane = threadIdx.x & 31;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nchunks; c += (gridDim.x * blockDim.x) >> 5) {
        const int4 d = desc[c];
        const int k0 = ptr[d.x], cnt = ptr[d.y] - k0;
        for (int e = lane; e < cnt; e += 32) {
            if (pidx) pidx[d.z + e] = idx[k0 + e];
            if (pval) pval[d.z + e] = T(val[k0 + e]);
        }
    }
}

// ------------------------------------------------------------------------------------ staged layout
// The staged sweeps' entry arrays (mfs_staged.cuh) from a device order (segment pointers ptr,
// gathered indices idx, FP64 values val): per group of segments, its entries in the order of
// (block of the gathered index, segment, gathered index) -- a stable split of the group's entries,
// which are already in (segment, gathered index) order, by block -- each 8-byte entry holding the
// segment's index within the group (low 16 bits), the gathered index within the block (high 16
// bits) and the FP32 value; then every warp's range laid out over its lanes (k_stg_lanes).

// segment of every entry: seg_of[k] = s for k in [ptr[s], ptr[s+1])
__global__ void k_seg_of(const int* __restrict__ ptr, int nseg, int* __restrict__ seg_of) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nseg; s += gridDim.x * blockDim.x)
        for (int k = ptr[s]; k < ptr[s + 1]; ++k) seg_of[k] = s;
}

// cnt[g * R + b]: entries of group g whose gathered index falls in block b (one CTA per group)
__global__ void k_stg_count(const int* __restrict__ ptr, const int* __restrict__ grp, const int* __restrict__ idx,
                            int R, int rb, int* __restrict__ cnt) {
    extern __shared__ int hist[];
    const int g = blockIdx.x;
    for (int b = threadIdx.x; b < R; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    const int k0 = ptr[grp[g]], k1 = ptr[grp[g + 1]];
    for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) atomicAdd(hist + idx[k] / rb, 1);
    __syncthreads();
    for (int b = threadIdx.x; b < R; b += blockDim.x) cnt[(size_t)g * R + b] = hist[b];
}

// Stable split of group g's entries by block (one CTA of SNT threads per group, entries taken
// SNT at a time in order): an entry's slot is its block's start, plus the entries of that block
// in earlier rounds, in earlier warps of this round, and in earlier lanes of its warp.
constexpr int SNT = 512;
__global__ void __launch_bounds__(SNT) k_stg_scatter(const int* __restrict__ ptr, const int* __restrict__ grp,
                                                     const int* __restrict__ seg_of, const int* __restrict__ idx,
                                                     const double* __restrict__ val, int R, int rb,
                                                     const int* __restrict__ bstart, int2* __restrict__ ent) {
    extern __shared__ int sm[];
    int* run = sm;              // R: entries of each block placed so far
    int* wc = sm + R;           // (SNT/32) x R: entries of each block per warp in this round
    const int g = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int s0 = grp[g];
    for (int b = threadIdx.x; b < R; b += SNT) run[b] = 0;
    const int k0 = ptr[s0], k1 = ptr[grp[g + 1]];
    for (int base = k0; base < k1; base += SNT) {
        for (int q = threadIdx.x; q < (SNT / 32) * R; q += SNT) wc[q] = 0;
        __syncthreads();
        const int k = base + threadIdx.x;
        const bool ok = k < k1;
        const int b = ok ? idx[k] / rb : -1 - lane;  // inactive lanes never match each other
        const unsigned peers = __match_any_sync(0xffffffffu, b);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (ok && rank == 0) wc[warp * R + b] = __popc(peers);
        __syncthreads();
        if (ok) {
            int before = 0;
            for (int w = 0; w < warp; ++w) before += wc[w * R + b];
            const int at = bstart[(size_t)g * R + b] + run[b] + before + rank;
            const int gi = idx[k] - b * rb;
            const float v = (float)val[k];
            ent[at] = make_int2((seg_of[k] - s0) | (gi << 16), __float_as_int(v));
        }
        __syncthreads();
        for (int bb = threadIdx.x; bb < R; bb += SNT) {
            int add = 0;
            for (int w = 0; w < SNT / 32; ++w) add += wc[w * R + bb];
            run[bb] += add;
        }
        __syncthreads();
    }
}

// Warp ranges of every (group, block): split[u * (NW1) + w] = first entry of bucket u whose segment
// is at or after wseg[g][w] (w = 0 .. NW1-1; the last one is the bucket's end).
__global__ void k_stg_split(const int2* __restrict__ ent, const int* __restrict__ bstart, const int* __restrict__ cnt,
                            const int* __restrict__ wseg, int R, int nbuckets, int NW1, int* __restrict__ split) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < nbuckets; u += gridDim.x * blockDim.x) {
        const int g = u / R, st = bstart[u], en = st + cnt[u];
        int* sp = split + (size_t)u * NW1;
        sp[0] = st;
        for (int w = 1; w < NW1 - 1; ++w) {
            const int key = wseg[g * NW1 + w];
            int lo = sp[w - 1], hi = en;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if ((ent[mid].x & 0xFFFF) < key)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            sp[w] = lo;
        }
        sp[NW1 - 1] = en;
    }
}

// Lane layout of every warp range (mfs_staged.cuh): the range [st, en) of a (group, block, warp)
// holds that warp's entries of the block in (segment, gathered index) order. With n entries it is
// laid out in R = ceil(n / 32) rounds, lanes l < n - 32 (R - 1) taking R entries and the others
// R - 1, lane l's entries at st + 32 r + l. Every run (the entries of one segment) goes to one lane,
// consecutive and in order: runs longer than LONGRUN first, in their order, then the runs of
// LONGRUN down to 2 entries, longest first, each into the lane with the most room left (the lowest
// such lane); a run longer than that room fills it and its rest goes on the same way, piece j > 0
// then adding into the segment's j-th overflow slot. Last, the single entries fill the lanes' room
// in lane order. Phase 0 records each segment's largest number of pieces over the blocks; phase 1
// writes the entries in place with their slots (the segment for piece 0, else its overflow slot).
// The same steps in both phases give the same placement.
constexpr int LONGRUN = 8;

template <int PHASE>
__global__ void k_stg_lanes(const int2* __restrict__ ent, const int* __restrict__ split, long long nranges, int NW1,
                            int R, const int* __restrict__ grp, int* __restrict__ npieces, const int* __restrict__ ovf,
                            int2* __restrict__ out) {
    for (long long rg = blockIdx.x * (long long)blockDim.x + threadIdx.x; rg < nranges;
         rg += (long long)gridDim.x * blockDim.x) {
        const long long u = rg / (NW1 - 1);
        const int w = (int)(rg % (NW1 - 1));
        const int st = split[u * NW1 + w], en = split[u * NW1 + w + 1], n = en - st;
        if (n <= 0) continue;
        const int s0 = grp[u / R];
        const int rounds = (n + 31) / 32, full = n - 32 * (rounds - 1);
        int cap[32], fill[32];
        for (int l = 0; l < 32; ++l) {
            cap[l] = l < full ? rounds : rounds - 1;
            fill[l] = 0;
        }
        auto seg_at = [&](int p) { return ent[p].x & 0xFFFF; };
        auto run_end = [&](int p) {
            const int sg = seg_at(p);
            int q = p + 1;
            while (q < en && seg_at(q) == sg) ++q;
            return q;
        };
        auto put = [&](int p, int lane, int slot) {
            if (PHASE == 1)
                out[st + fill[lane] * 32 + lane] = make_int2((ent[p].x & (int)0xFFFF0000) | slot, ent[p].y);
            --cap[lane];
            ++fill[lane];
        };
        auto place = [&](int p, int len) {
            const int sg = seg_at(p);
            int j = 0;
            while (len > 0) {
                int best = 0;
                for (int l = 1; l < 32; ++l)
                    if (cap[l] > cap[best]) best = l;
                const int t = len < cap[best] ? len : cap[best];
                const int slot = j == 0 ? sg : (PHASE == 1 ? ovf[s0 + sg] + j - 1 : 0);
                for (int i = 0; i < t; ++i) put(p + i, best, slot);
                p += t;
                len -= t;
                ++j;
            }
            if (PHASE == 0 && j > 1) atomicMax(npieces + s0 + sg, j);
        };
        for (int p = st; p < en;) {  // long runs, in order
            const int q = run_end(p);
            if (q - p > LONGRUN) place(p, q - p);
            p = q;
        }
        for (int L = LONGRUN; L >= 2; --L)  // shorter runs, longest first
            for (int p = st; p < en;) {
                const int q = run_end(p);
                if (q - p == L) place(p, L);
                p = q;
            }
        int lane = 0;  // single entries, lanes in order
        for (int p = st; p < en;) {
            const int q = run_end(p);
            if (q - p == 1) {
                while (cap[lane] == 0) ++lane;
                put(p, lane, seg_at(p));
            }
            p = q;
        }
    }
}

// Overflow slots, from the largest number of pieces of each segment over the blocks (npieces; 0 or
// 1: none). c1[s] = the segment's overflow slots, c2[s] = 1 if it has any; their exclusive scans
// (device-wide, so over all groups at once) place everything: a group's overflow slots follow its
// segments, allocated in segment order, so that each warp's are contiguous.
__global__ void k_stg_ovf_counts(const int* __restrict__ npieces, int nseg, int* __restrict__ c1, int* __restrict__ c2) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nseg; t += gridDim.x * blockDim.x) {
        const int np = npieces[t];
        c1[t] = np > 1 ? np - 1 : 0;
        c2[t] = np > 1 ? 1 : 0;
    }
}

// group of segment s: the last g with grp[g] <= s
__device__ __forceinline__ int group_of(const int* __restrict__ grp, int G, int s) {
    int lo = 0, hi = G;  // grp[lo] <= s < grp[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (grp[mid] <= s) lo = mid; else hi = mid;
    }
    return lo;
}

// Per segment with overflow slots: ovf[s] = its first overflow slot within the group (s1, s2: the
// exclusive scans of c1, c2, each with its total at index nseg) and its fold entry
// (segment within the group, first overflow slot | (pieces - 1) << 16) at position s2[s].
__global__ void k_stg_ovf_place(const int* __restrict__ grp, int G, const int* __restrict__ npieces,
                                const int* __restrict__ s1, const int* __restrict__ s2, int nseg,
                                int* __restrict__ ovf, int2* __restrict__ fold) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nseg; t += gridDim.x * blockDim.x) {
        const int np = npieces[t];
        if (np <= 1) continue;
        const int g = group_of(grp, G, t), a = grp[g];
        const int slot = (grp[g + 1] - a) + (s1[t] - s1[a]);
        ovf[t] = slot;
        fold[s2[t]] = make_int2(t - a, slot | ((np - 1) << 16));
    }
}

// Per (group, warp): its first overflow slot (wovf, G x NW1, the last one the group's end) and the
// start of its fold entries (fold_ptr, G * (NW1 - 1) + 1); *slots_max = the largest group's slots.
__global__ void k_stg_ovf_warps(const int* __restrict__ grp, int G, const int* __restrict__ wseg, int NW1,
                                const int* __restrict__ s1, const int* __restrict__ s2, int nseg,
                                int* __restrict__ wovf, int* __restrict__ fold_ptr, int* __restrict__ slots_max) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < G * NW1; q += gridDim.x * blockDim.x) {
        const int g = q / NW1, w = q % NW1, a = grp[g], nseg_g = grp[g + 1] - a;
        const int at = a + wseg[q];
        wovf[q] = nseg_g + (s1[at] - s1[a]);
        if (w < NW1 - 1) fold_ptr[g * (NW1 - 1) + w] = s2[at];
        if (w == NW1 - 1) atomicMax(slots_max, nseg_g + (s1[at] - s1[a]));
        if (q == 0) fold_ptr[G * (NW1 - 1)] = s2[nseg];
    }
}

// 1/(1 + r_i) of each row, r_i the sum of the squared FP32-rounded values of row i: in FP64, rounded
// to FP32 (the staged row pass multiplies by it)
__global__ void k_row_inv(const int* __restrict__ row_ptr, const double* __restrict__ val, int m,
                          float* __restrict__ rinv) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        double r = 0.0;
        for (int k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            const double a = (double)(float)val[k];
            r += a * a;
        }
        rinv[i] = (float)(1.0 / (1.0 + r));
    }
}

// 1/(1 + d_j) of each column, d_j its number of nonzeros, rounded to FP32 (the staged column pass
// multiplies by it)
__global__ void k_col_inv(const int* __restrict__ col_ptr, int n, float* __restrict__ dinv) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        dinv[j] = (float)(1.0 / (1.0 + (double)(col_ptr[j + 1] - col_ptr[j])));
}

}  // namespace setup
}  // namespace mfs
