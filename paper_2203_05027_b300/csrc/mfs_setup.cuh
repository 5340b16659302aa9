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
// whether some entry comes before its predecessor in (column, row) order.
__global__ void k_check(const long long* __restrict__ row, const long long* __restrict__ col,
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

// In column order (duplicates allowed): keep[q] = 1 where a run of equal (column, row) starts and
// its values sum to a nonzero, sum[q] = that sum (in entry order).
__global__ void k_runs(const long long* __restrict__ row, const long long* __restrict__ col,
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

__global__ void k_compact(const long long* __restrict__ row, const long long* __restrict__ col,
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

}  // namespace setup
}  // namespace mfs
