// mfs_solver.cu -- host side of libmfs: problem set-up (Algorithm 1, steps 1-3), device memory,
// the iteration driver (CUDA graphs of whole check intervals), residuals, precision switching and
// the C ABI declared in include/mfs.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <limits>
#include <mutex>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/mfs.h"
#include "mfs_alloc.h"
#include "mfs_host.h"
#include "mfs_kernels.cuh"
#include "mfs_staged.cuh"
#include "mfs_infeas.cuh"
#include "mfs_literal.cuh"
#include "mfs_measures.h"
#include "mfs_trace.h"
#include "mfs_setup.cuh"

using namespace mfs;

using StagedArgsT = mfs::staged::StagedArgs;

namespace {

thread_local std::string g_create_error;

template <typename T>
struct State {
    T* x = nullptr;
    T* z = nullptr;
    T* del = nullptr;
    T* lam = nullptr;
    T* v = nullptr;
    T* b = nullptr;
    T* c = nullptr;
    T* cval = nullptr;
    T* rval = nullptr;
    cudaGraphExec_t graph = nullptr;  // check_every iterations
    int graph_iters = 0;
};

using mfs::host::Chunks;

// Both orders of A built on the GPU (device set-up), kept until the padded layouts are filled.
struct DevOrders {
    bool on = false;
    int *crow = nullptr, *rcol = nullptr;     // row indices in column order, column indices in row order
    double *cval = nullptr, *rval = nullptr;  // the values in both orders
    std::vector<void*> mem;                   // everything this set-up allocated
    ~DevOrders() {
        for (void* q : mem) cudaFree(q);
    }
};

struct HostProblem {
    int m = 0, n = 0, o = 0;
    std::vector<int> col_ptr, row_ptr;
    DevOrders dev;                    // on: the unpadded orders live on the device only
    mfs::host::uvec<int> csc_row;     // unpadded, column order
    mfs::host::uvec<double> csc_val;
    mfs::host::uvec<int> csr_col;     // unpadded, row order
    mfs::host::uvec<double> csr_val;
    Chunks cc, rc;
    std::vector<int> cq_lo, cq_hi;
    std::vector<int> soc_start, soc_size, big_list;
    std::vector<unsigned char> soc_big;
};

}  // namespace

struct mfs_solver {
    int device = 0;
    cudaStream_t stream = nullptr;   // where the caller's work is ordered
    cudaStream_t cap = nullptr;      // private stream used only to capture graphs
    bool own_stream = false;
    mfs_settings set{};
    int precision = MFS_FP64;        // precision the iterate is held in now
    int64_t iter = 0;
    int m = 0, n = 0, o = 0;
    int ncones = 0, nsoc = 0, nbig = 0;
    int ncc = 0, nrc = 0;            // column / row chunks
    long long cpad = 0, rpad = 0;    // lengths of the padded column / row nonzero arrays
    int nlc = 0, nlr = 0;            // long column / row chunks
    bool has_soc = false;
    int num_sms = 148;
    int g_rowres = 1, g_colres = 1;  // persistent residual grids
    // shared device structure
    int *col_ptr = nullptr, *cidx = nullptr, *cq_lo = nullptr, *cq_hi = nullptr, *clong = nullptr;
    int *row_ptr = nullptr, *ridx = nullptr, *rlong = nullptr;
    uint32_t *cheads = nullptr, *rheads = nullptr;
    int4 *cdesc = nullptr, *rdesc = nullptr;
    int *soc_start = nullptr, *soc_size = nullptr, *big_list = nullptr;
    unsigned char* soc_big = nullptr;
    int* stg_big_list = nullptr;  // the staged column pass fuses every cone of at most WC columns;
    int stg_nbig = 0;             // these are the larger ones, left to k_bigcone_sweep
    double *part_row = nullptr, *part_col = nullptr, *part_big = nullptr, *s_buf = nullptr, *status = nullptr;
    double* r_buf = nullptr;  // m: A x - b of the last residual evaluation with write_all_s
    double* h_status = nullptr;      // pinned
    State<float> s32;
    State<double> s64;
    bool have32 = false, have64 = false;
    // literal start (Algorithm 1 with o-length y and gamma) pending for the next lit_pending iterations
    int lit_pending = 0;
    // primal infeasibility test of mfs_solve: previous s = c + A^T lambda and lambda (FP64)
    unsigned char* in_cone = nullptr;  // n: 0 orthant, 1 small Lorentz cone, 2 Lorentz cone of the big-cone kernels
    double *inf_s_prev = nullptr, *inf_lam_prev = nullptr, *inf_x_prev = nullptr, *inf_r_prev = nullptr,
           *inf_part = nullptr;
    void *lit_y = nullptr, *lit_g = nullptr, *lit_kval = nullptr, *lit_w = nullptr, *lit_row = nullptr;
    int *lit_krow = nullptr, *lit_kcol = nullptr, *lit_perm = nullptr, *lit_rp = nullptr;
    double* lit_zarg = nullptr;
    std::vector<void*> lit_mem;
    // checks of the last mfs_solve, oldest first once the ring has wrapped (hist_next = next slot)
    std::vector<mfs_check_t> hist;
    int64_t hist_count = 0;
    // staged FP32 sweeps (mfs_staged.cuh): built at create for FP32 problems without Lorentz cones
    bool stg_ok = false;
    bool stg_auto_col = false;  // the automatic choice runs the staged column pass
    bool stg_auto_row = false;  // the automatic choice runs the staged row pass
    int sweep_kind = MFS_SWEEP_AUTO;
    mfs::staged::StagedArgs stg_col{}, stg_row{};
    bool keep_l2 = false;  // holds a reference on the raised persisting-L2 limit (settings.l2_keep)
    int* stg_err = nullptr;
    int* h_err = nullptr;  // pinned
    std::vector<void*> allocs;
    std::string last_error;
};

namespace {

mfs_status fail(mfs_solver* s, mfs_status st, const std::string& msg) {
    if (s)
        s->last_error = msg;
    else
        g_create_error = msg;
    return st;
}

#define CUDA_TRY(s, call)                                                                          \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail((s), e_ == cudaErrorMemoryAllocation ? MFS_ERR_OOM : MFS_ERR_CUDA,          \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                       \
    } while (0)

#define TRY(x)                               \
    do {                                     \
        mfs_status st_ = (x);                \
        if (st_ != MFS_OK) return st_;       \
    } while (0)

template <typename T>
mfs_status dalloc(mfs_solver* s, T** p, size_t count) {
    void* q = nullptr;
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = mfs::device_malloc(&q, bytes);
    if (e != cudaSuccess)
        return fail(s, e == cudaErrorMemoryAllocation ? MFS_ERR_OOM : MFS_ERR_CUDA,
                    std::string("cudaMalloc: ") + cudaGetErrorString(e));
    s->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return MFS_OK;
}

template <typename T>
mfs_status upload(mfs_solver* s, T** p, const void* host, size_t count) {
    TRY(dalloc(s, p, count));
    if (count) CUDA_TRY(s, cudaMemcpyAsync(*p, host, count * sizeof(T), cudaMemcpyHostToDevice, s->stream));
    return MFS_OK;
}

// ---------------------------------------------------------------------------------- host set-up

// Sort COO into column order (rows ascending within a column), sum duplicates, drop zeros;
// then build the row order (columns ascending within a row). Stable counting sorts, O(nnz + m + n),
// multi-threaded (mfs_host.h); an input already in strict column order skips the sorting.
// in_order: the caller found the input in (column, row) order, duplicates next to each other.
void build_orders(int64_t m, int64_t n, int64_t nnz, const int64_t* row, const int64_t* col, const double* val,
                  bool in_order, HostProblem& P) {
    using namespace mfs::host;
    const int nt = threads_for(nnz);
    // order of the input entries by (column, row)
    uvec<int64_t> ord((size_t)nnz);
    if (in_order) {
        parallel_ranges(nnz, nt, [&](int64_t lo, int64_t hi, int) {
            for (int64_t q = lo; q < hi; ++q) ord[q] = q;
        });
    } else {
        uvec<int64_t> by_row((size_t)nnz);
        counting_sort(nnz, m, [&](int64_t q) { return row[q]; }, nullptr, by_row.data(), nullptr);
        counting_sort(nnz, n, [&](int64_t q) { return col[by_row[q]]; }, by_row.data(), ord.data(), nullptr);
    }
    // sum duplicates and drop zeros: each thread compacts a range of groups of equal (column, row)
    std::vector<int64_t> cut(nt + 1, nnz);
    cut[0] = 0;
    for (int t = 1; t < nt; ++t) {
        int64_t q = nnz * t / nt;
        if (q < cut[t - 1]) q = cut[t - 1];
        while (q > 0 && q < nnz && row[ord[q]] == row[ord[q - 1]] && col[ord[q]] == col[ord[q - 1]]) ++q;
        cut[t] = q;
    }
    std::vector<uvec<int>> krow(nt), kcol(nt);
    std::vector<uvec<double>> kval(nt);
    parallel_tasks(nt, [&](int t) {
        // thread-local output with raw-pointer writes (no shared vector headers written per entry)
        const int64_t len = cut[t + 1] - cut[t];
        uvec<int> lr(len), lc(len);
        uvec<double> lv(len);
        int* pr = lr.data();
        int* pc = lc.data();
        double* pv = lv.data();
        int64_t w = 0, q = cut[t];
        while (q < cut[t + 1]) {
            const int64_t e = ord[q];
            const int64_t i = row[e], j = col[e];
            double a = val[e];
            ++q;
            while (q < cut[t + 1] && row[ord[q]] == i && col[ord[q]] == j) a += val[ord[q++]];
            if (a != 0.0) {
                pr[w] = (int)i;
                pc[w] = (int)j;
                pv[w] = a;
                ++w;
            }
        }
        lr.resize(w);
        lc.resize(w);
        lv.resize(w);
        krow[t] = std::move(lr);
        kcol[t] = std::move(lc);
        kval[t] = std::move(lv);
    });
    ord.clear();
    ord.shrink_to_fit();
    std::vector<int64_t> off(nt + 1, 0);
    for (int t = 0; t < nt; ++t) off[t + 1] = off[t] + (int64_t)krow[t].size();
    const int64_t o = off[nt];
    P.m = (int)m;
    P.n = (int)n;
    P.o = (int)o;
    P.csc_row.resize(o);
    P.csc_val.resize(o);
    uvec<int> ccol(o);
    parallel_tasks(nt, [&](int t) {
        {
            std::copy(krow[t].begin(), krow[t].end(), P.csc_row.begin() + off[t]);
            std::copy(kval[t].begin(), kval[t].end(), P.csc_val.begin() + off[t]);
            std::copy(kcol[t].begin(), kcol[t].end(), ccol.begin() + off[t]);
            uvec<int>().swap(krow[t]);
            uvec<int>().swap(kcol[t]);
            uvec<double>().swap(kval[t]);
        }
    });
    // column pointers: entries are in column order, so col_ptr[j] is the first entry of a column >= j
    P.col_ptr.resize(n + 1);
    parallel_ranges(o, threads_for(o), [&](int64_t lo, int64_t hi, int) {
        for (int64_t k = lo; k < hi; ++k)
            for (int j = (k ? ccol[k - 1] : -1) + 1; j <= ccol[k]; ++j) P.col_ptr[j] = (int)k;
    });
    for (int64_t j = (o ? ccol[o - 1] + 1 : 0); j <= n; ++j) P.col_ptr[j] = (int)o;
    // row order from column order: stable by k, so columns ascend within a row
    uvec<int64_t> by_row((size_t)o);
    std::vector<int64_t> rstart;
    counting_sort(o, m, [&](int64_t k) { return (int64_t)P.csc_row[k]; }, nullptr, by_row.data(), &rstart);
    P.row_ptr.resize(m + 1);
    for (int64_t i = 0; i <= m; ++i) P.row_ptr[i] = (int)rstart[i];
    P.csr_col.resize(o);
    P.csr_val.resize(o);
    parallel_ranges(o, threads_for(o), [&](int64_t lo, int64_t hi, int) {
        for (int64_t p = lo; p < hi; ++p) {
            const int64_t k = by_row[p];
            P.csr_col[p] = ccol[k];
            P.csr_val[p] = P.csc_val[k];
        }
    });
}

// Plan of one staged pass (mfs_staged.cuh), made on the host.
struct StagedHost {
    std::vector<int> grp, wseg;
    int G = 0, R = 0, maxg = 0;
};

// Plan of a staged pass: segments (columns, or rows) in groups of consecutive segments balanced by
// nonzeros (nominally `groups`, at most MAXG segments each, and as many as the shared memory left
// by the stages and split table holds), and each warp's segments within its group, balanced by
// nonzeros. rb: entries of the gathered vector per block. Returns false if not even small groups
// fit. The entries themselves are laid out on the GPU (staged_on_device).
bool plan_staged(const std::vector<int>& ptr, int nseg, int nother, int groups, int rb, int stages,
                 size_t smem_limit, StagedHost& S, const std::vector<int>* unit_start = nullptr) {
    // a boundary never falls inside a unit (a small Lorentz cone, whose columns one warp projects)
    auto snap = [&](int b) { return (unit_start && b > 0 && b < nseg) ? (*unit_start)[b] : b; };
    using mfs::staged::NW;
    const int RB = rb;
    const int64_t o = ptr[nseg];
    S.R = std::max(1, (nother + RB - 1) / RB);
    const size_t fixed = mfs::staged::smem_bytes(RB, stages, 0, S.R);
    if (fixed + 4096 * 4 > smem_limit) return false;
    const int MAXG = (int)std::min<size_t>(mfs::staged::MAXG, (smem_limit - fixed) / 16 * 4);
    S.grp.assign(1, 0);
    int lo = 0;
    for (int g = 1; g <= groups; ++g) {
        int hi = nseg;
        if (g < groups) {
            const int target = (int)(o * g / groups);
            hi = (int)(std::lower_bound(ptr.begin(), ptr.begin() + nseg + 1, target) - ptr.begin());
            hi = std::min(std::max(snap(hi), lo), nseg);
        }
        while (hi - lo > MAXG) {
            lo = snap(lo + MAXG);
            S.grp.push_back(lo);
        }
        if (hi > lo) {
            S.grp.push_back(hi);
            lo = hi;
        }
    }
    if (S.grp.size() == 1) S.grp.push_back(nseg);
    S.G = (int)S.grp.size() - 1;
    S.maxg = 0;
    for (int g = 0; g < S.G; ++g) S.maxg = std::max(S.maxg, S.grp[g + 1] - S.grp[g]);
    const int G = S.G;
    S.wseg.resize((size_t)G * (NW + 1));
    for (int g = 0; g < G; ++g) {
        const int a = S.grp[g], e = S.grp[g + 1];
        const int64_t nz = (int64_t)ptr[e] - ptr[a];
        int* w = S.wseg.data() + (size_t)g * (NW + 1);
        w[0] = 0;
        for (int q = 1; q < NW; ++q) {
            const int target = (int)(ptr[a] + nz * q / NW);
            const int at = (int)(std::lower_bound(ptr.begin() + a, ptr.begin() + e + 1, target) - ptr.begin());
            w[q] = std::max(w[q - 1], std::max(snap(std::min(at, e)), a) - a);
        }
        w[NW] = e - a;
    }
    return true;
}

// Exclusive scan of n ints on the device (mfs_setup.cuh); *total (nullable) receives their sum.
mfs_status device_scan(mfs_solver* s, const int* in, int* out, int64_t n, int* total) {
    namespace su = mfs::setup;
    if (n <= 0) {
        if (total) *total = 0;
        return MFS_OK;
    }
    const int blocks = (int)((n + su::SPAN - 1) / su::SPAN);
    int* blk = nullptr;
    cudaError_t e = mfs::device_malloc((void**)&blk, (size_t)(blocks + 1) * sizeof(int));
    if (e != cudaSuccess) return fail(s, MFS_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    su::k_scan_local<<<blocks, su::NT, 0, s->stream>>>(in, out, blk, n);
    su::k_scan_blocks<<<1, 1024, 0, s->stream>>>(blk, blocks, blk + blocks);
    su::k_scan_add<<<blocks, su::NT, 0, s->stream>>>(out, blk, n);
    if (total) cudaMemcpyAsync(total, blk + blocks, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
    cudaStreamSynchronize(s->stream);
    cudaFree(blk);
    CUDA_TRY(s, cudaGetLastError());
    return MFS_OK;
}

// Device set-up (mfs_setup.cuh): upload the COO, check it, and if it is valid and in column order
// (duplicates next to each other) build both orders on the GPU, leaving P.dev.on set and P.col_ptr, P.row_ptr, P.o on the host.
// An input out of order leaves P.dev.on unset (the host orders it); an invalid one fails.
// Host-to-device copies of large pageable arrays through pinned staging buffers: each of up to 16
// host threads takes its slice of every array and fills its two 2 MB buffers in turn while the copy
// engine drains the other on the thread's own stream; `st` then waits for all of them. An array of
// int64 indices with a limit is narrowed to int32 on the way, each index checked against
// [0, limit) first. The buffers and streams belong to the process (one set, for the device that
// first used it, taken under a lock); any other device, or a failure to set them up, gets copies
// from pageable memory.
struct PinnedStaging {
    std::mutex mu;
    int device = -1;  // -2: unavailable
    int nt = 0;
    static constexpr size_t SUB = size_t(2) << 20;
    std::vector<char*> buf;         // 2 per thread
    std::vector<cudaStream_t> str;  // 1 per thread
    std::vector<cudaEvent_t> ev;    // 2 per thread, + 1 per thread marking its last copy
    cudaEvent_t ready = nullptr;    // downloads: the source is complete on the caller's stream
};
static PinnedStaging g_pin;

struct HostCopy {
    void* dst;
    const void* src;
    size_t bytes;      // at the source
    int64_t lim = 0;   // > 0: src holds bytes / 8 int64 indices, sent as int32, each checked against [0, lim)
};

static bool pinned_ready(int device) {
    if (g_pin.device == device) return true;
    if (g_pin.device != -1) return false;
    g_pin.device = -2;
    const unsigned h = std::thread::hardware_concurrency();
    const int nt = (int)std::max(1u, std::min(h ? h : 1u, 16u));
    for (int t = 0; t < nt; ++t) {
        cudaStream_t q = nullptr;
        if (cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking) != cudaSuccess) return false;
        g_pin.str.push_back(q);
        for (int k = 0; k < 3; ++k) {
            cudaEvent_t e = nullptr;
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return false;
            g_pin.ev.push_back(e);
        }
    }
    void* block = nullptr;  // one pinned allocation, cut into two buffers per thread
    if (cudaHostAlloc(&block, 2 * (size_t)nt * PinnedStaging::SUB, cudaHostAllocDefault) != cudaSuccess) return false;
    for (int b = 0; b < 2 * nt; ++b) g_pin.buf.push_back(static_cast<char*>(block) + b * PinnedStaging::SUB);
    if (cudaEventCreateWithFlags(&g_pin.ready, cudaEventDisableTiming) != cudaSuccess) return false;
    g_pin.nt = nt;
    g_pin.device = device;
    return true;
}

// *first_bad: the first position (in any index array) with an index out of range, or SIZE_MAX.
mfs_status upload_pinned(mfs_solver* s, const std::vector<HostCopy>& copies, cudaStream_t st, size_t* first_bad) {
    std::lock_guard<std::mutex> lock(g_pin.mu);
    *first_bad = SIZE_MAX;
    if (!pinned_ready(s->device)) {
        cudaGetLastError();  // a failed set-up leaves nothing behind; copy from pageable memory
        for (const HostCopy& c : copies) {
            if (c.lim > 0) {
                const size_t n = c.bytes / 8;
                std::vector<int32_t> tmp(n);
                const size_t bad = mfs::host::narrow_indices(static_cast<const int64_t*>(c.src), tmp.data(), n, c.lim);
                if (bad < n) *first_bad = std::min(*first_bad, bad);
                CUDA_TRY(s, cudaMemcpyAsync(c.dst, tmp.data(), n * 4, cudaMemcpyHostToDevice, st));
                CUDA_TRY(s, cudaStreamSynchronize(st));  // tmp goes out of scope
            } else {
                CUDA_TRY(s, cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyHostToDevice, st));
            }
        }
        return MFS_OK;
    }
    const int T = g_pin.nt;
    std::vector<cudaError_t> err(T, cudaSuccess);
    std::vector<size_t> bad(T, SIZE_MAX);
    mfs::host::parallel_tasks(T, [&](int t) {
        cudaError_t e = cudaSetDevice(s->device);
        int k = 0;
        for (const HostCopy& c : copies) {
            const bool idx = c.lim > 0;
            const size_t nel = idx ? c.bytes / 8 : c.bytes;  // elements (bytes for a plain copy)
            const size_t per = idx ? PinnedStaging::SUB / 4 : PinnedStaging::SUB;
            const size_t lo = nel * t / T, hi = nel * (t + 1) / T;
            for (size_t off = lo; off < hi && e == cudaSuccess; off += per) {
                const size_t len = std::min(per, hi - off);
                const int b = 2 * t + (k & 1);
                if (k >= 2) e = cudaEventSynchronize(g_pin.ev[3 * t + (k & 1)]);  // its previous copy is done
                if (e != cudaSuccess) break;
                if (idx) {
                    int32_t* bp = reinterpret_cast<int32_t*>(g_pin.buf[b]);
                    const size_t q = mfs::host::narrow_indices(static_cast<const int64_t*>(c.src) + off, bp, len, c.lim);
                    if (q < len) bad[t] = std::min(bad[t], off + q);
                    e = cudaMemcpyAsync(static_cast<int32_t*>(c.dst) + off, bp, len * 4, cudaMemcpyHostToDevice,
                                        g_pin.str[t]);
                } else {
                    std::memcpy(g_pin.buf[b], static_cast<const char*>(c.src) + off, len);
                    e = cudaMemcpyAsync(static_cast<char*>(c.dst) + off, g_pin.buf[b], len, cudaMemcpyHostToDevice,
                                        g_pin.str[t]);
                }
                if (e == cudaSuccess) e = cudaEventRecord(g_pin.ev[3 * t + (k & 1)], g_pin.str[t]);
                ++k;
            }
        }
        if (e == cudaSuccess) e = cudaEventRecord(g_pin.ev[3 * t + 2], g_pin.str[t]);
        err[t] = e;
    });
    for (int t = 0; t < T; ++t) CUDA_TRY(s, err[t]);
    for (int t = 0; t < T; ++t) *first_bad = std::min(*first_bad, bad[t]);
    for (int t = 0; t < T; ++t) CUDA_TRY(s, cudaStreamWaitEvent(st, g_pin.ev[3 * t + 2], 0));
    // the buffers are reused by the next upload: let these copies finish first
    for (int t = 0; t < T; ++t) CUDA_TRY(s, cudaEventSynchronize(g_pin.ev[3 * t + 2]));
    return MFS_OK;
}

// Device-to-host copies into pageable arrays, the reverse of upload_pinned: each thread issues the
// copy of its next piece into one of its buffers while it moves the previous piece out of the other.
// Returns when every byte has reached the host.
mfs_status download_pinned(mfs_solver* s, const std::vector<HostCopy>& copies, cudaStream_t st) {
    std::lock_guard<std::mutex> lock(g_pin.mu);
    if (!pinned_ready(s->device)) {
        cudaGetLastError();
        for (const HostCopy& c : copies)
            CUDA_TRY(s, cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(s, cudaStreamSynchronize(st));
        return MFS_OK;
    }
    CUDA_TRY(s, cudaEventRecord(g_pin.ready, st));
    const int T = g_pin.nt;
    std::vector<cudaError_t> err(T, cudaSuccess);
    mfs::host::parallel_tasks(T, [&](int t) {
        cudaError_t e = cudaSetDevice(s->device);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(g_pin.str[t], g_pin.ready, 0);
        char* pend = nullptr;  // host destination of the piece in flight in buffer (k - 1) & 1
        size_t plen = 0;
        int k = 0;
        auto drain = [&](int kk) {  // move piece kk (already issued) out of its buffer
            if (e == cudaSuccess) e = cudaEventSynchronize(g_pin.ev[3 * t + (kk & 1)]);
            if (e == cudaSuccess) std::memcpy(pend, g_pin.buf[2 * t + (kk & 1)], plen);
        };
        for (const HostCopy& c : copies) {
            const size_t lo = c.bytes * t / T, hi = c.bytes * (t + 1) / T;
            for (size_t off = lo; off < hi && e == cudaSuccess; off += PinnedStaging::SUB) {
                const size_t len = std::min(PinnedStaging::SUB, hi - off);
                const int b = 2 * t + (k & 1);
                e = cudaMemcpyAsync(g_pin.buf[b], static_cast<const char*>(c.src) + off, len, cudaMemcpyDeviceToHost,
                                    g_pin.str[t]);
                if (e == cudaSuccess) e = cudaEventRecord(g_pin.ev[3 * t + (k & 1)], g_pin.str[t]);
                if (k >= 1) drain(k - 1);
                pend = static_cast<char*>(c.dst) + off;
                plen = len;
                ++k;
            }
        }
        if (k >= 1) drain(k - 1);
        err[t] = e;
    });
    for (int t = 0; t < T; ++t) CUDA_TRY(s, err[t]);
    return MFS_OK;
}

// COO on the host (uploaded here) or, with on_device, already in device memory. Returns MFS_OK with
// P.dev.on false when the entries are not in column order (the host orders them then).
mfs_status device_orders(mfs_solver* s, int64_t m, int64_t n, int64_t nnz, const int64_t* row, const int64_t* col,
                         const double* val, HostProblem& P, bool on_device = false) {
    namespace su = mfs::setup;
    DevOrders& D = P.dev;
    auto grab = [&](void** q, size_t bytes) -> mfs_status {
        cudaError_t e = mfs::device_malloc(q, std::max<size_t>(bytes, 16));
        if (e != cudaSuccess)
            return fail(s, e == cudaErrorMemoryAllocation ? MFS_ERR_OOM : MFS_ERR_CUDA,
                        std::string("cudaMalloc: ") + cudaGetErrorString(e));
        D.mem.push_back(*q);
        return MFS_OK;
    };
    cudaStream_t st = s->stream;
    const int grid = 8 * s->num_sms;
    int *d_row = nullptr, *d_col = nullptr;
    double *d_val = nullptr, *d_sum = nullptr;
    int *d_keep = nullptr, *d_pos = nullptr, *d_flags = nullptr;
    unsigned long long* d_bad = nullptr;
    TRY(grab((void**)&d_row, nnz * sizeof(int)));
    TRY(grab((void**)&d_col, nnz * sizeof(int)));
    TRY(grab((void**)&d_bad, 2 * sizeof(unsigned long long) + 2 * sizeof(int)));
    d_flags = reinterpret_cast<int*>(d_bad + 2);
    size_t bad_host = SIZE_MAX;  // first entry with an index out of range, found while narrowing
    if (on_device) {
        d_val = const_cast<double*>(val);  // only read
        su::k_narrow_dev<<<grid, su::NT, 0, st>>>(reinterpret_cast<const long long*>(row), nnz, m, d_row);
        su::k_narrow_dev<<<grid, su::NT, 0, st>>>(reinterpret_cast<const long long*>(col), nnz, n, d_col);
        CUDA_TRY(s, cudaGetLastError());
    } else {
        TRY(grab((void**)&d_val, nnz * sizeof(double)));
        TRY(upload_pinned(s, {{d_row, row, nnz * sizeof(int64_t), m}, {d_col, col, nnz * sizeof(int64_t), n},
                              {d_val, val, nnz * sizeof(double)}}, st, &bad_host));
    }
    {
        unsigned long long init[2] = {(unsigned long long)nnz, (unsigned long long)nnz};
        CUDA_TRY(s, cudaMemcpyAsync(d_bad, init, sizeof init, cudaMemcpyHostToDevice, st));
        CUDA_TRY(s, cudaMemsetAsync(d_flags, 0, 2 * sizeof(int), st));
        su::k_check<<<grid, su::NT, 0, st>>>(d_row, d_col, d_val, nnz, m, n, d_bad, d_bad + 1, d_flags);
        unsigned long long bad[2];
        int flags[2];
        CUDA_TRY(s, cudaMemcpyAsync(bad, d_bad, sizeof bad, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(s, cudaMemcpyAsync(flags, d_flags, sizeof flags, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(s, cudaStreamSynchronize(st));
        const int64_t bi = std::min((int64_t)bad[0], bad_host < (size_t)nnz ? (int64_t)bad_host : nnz), bv = (int64_t)bad[1];
        if (bi < nnz && bi <= bv)
            return fail(s, MFS_ERR_INVALID, "COO index out of range at entry " + std::to_string(bi));
        if (bv < nnz) return fail(s, MFS_ERR_INVALID, "non-finite value in A");
        if (flags[0]) return MFS_OK;  // not in column order: the host sorts it
    }
    // runs of equal (column, row) summed, zero sums dropped, the rest compacted in order
    TRY(grab((void**)&d_keep, nnz * sizeof(int)));
    TRY(grab((void**)&d_pos, nnz * sizeof(int)));
    TRY(grab((void**)&d_sum, nnz * sizeof(double)));
    su::k_runs<<<grid, su::NT, 0, st>>>(d_row, d_col, d_val, nnz, d_keep, d_sum);
    int o = 0;
    TRY(device_scan(s, d_keep, d_pos, nnz, &o));
    int* d_ccol = nullptr;
    TRY(grab((void**)&D.crow, (size_t)o * sizeof(int)));
    TRY(grab((void**)&d_ccol, (size_t)o * sizeof(int)));
    TRY(grab((void**)&D.cval, (size_t)o * sizeof(double)));
    su::k_compact<<<grid, su::NT, 0, st>>>(d_row, d_col, d_keep, d_pos, d_sum, nnz, D.crow, d_ccol, D.cval);
    // column pointers; the row order by count, scan, scatter and a sort of each row by column
    int *d_cptr = nullptr, *d_rptr = nullptr, *d_cnt = nullptr;
    TRY(grab((void**)&d_cptr, (size_t)(n + 1) * sizeof(int)));
    TRY(grab((void**)&d_rptr, (size_t)(m + 1) * sizeof(int)));
    TRY(grab((void**)&d_cnt, (size_t)std::max<int64_t>(m, 1) * sizeof(int)));
    TRY(grab((void**)&D.rcol, (size_t)o * sizeof(int)));
    TRY(grab((void**)&D.rval, (size_t)o * sizeof(double)));
    CUDA_TRY(s, cudaMemsetAsync(d_cptr, 0, (size_t)(n + 1) * sizeof(int), st));
    if (o > 0) su::k_seg_ptr<<<grid, su::NT, 0, st>>>(d_ccol, o, (int)n, d_cptr);
    CUDA_TRY(s, cudaMemsetAsync(d_cnt, 0, (size_t)std::max<int64_t>(m, 1) * sizeof(int), st));
    su::k_count<<<grid, su::NT, 0, st>>>(D.crow, o, d_cnt);
    TRY(device_scan(s, d_cnt, d_rptr, m, nullptr));
    CUDA_TRY(s, cudaMemcpyAsync(d_rptr + m, &o, sizeof(int), cudaMemcpyHostToDevice, st));
    CUDA_TRY(s, cudaMemsetAsync(d_cnt, 0, (size_t)std::max<int64_t>(m, 1) * sizeof(int), st));
    su::k_scatter_rows<<<grid, su::NT, 0, st>>>(D.crow, d_ccol, D.cval, o, d_rptr, d_cnt, D.rcol, D.rval);
    if (m > 0) su::k_sort_rows<<<(int)std::min<int64_t>((m + su::NT - 1) / su::NT, grid), su::NT, 0, st>>>(d_rptr, (int)m, D.rcol, D.rval);
    CUDA_TRY(s, cudaGetLastError());
    P.m = (int)m;
    P.n = (int)n;
    P.o = o;
    P.col_ptr.resize(n + 1);
    P.row_ptr.resize(m + 1);
    CUDA_TRY(s, cudaMemcpyAsync(P.col_ptr.data(), d_cptr, (size_t)(n + 1) * sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(s, cudaMemcpyAsync(P.row_ptr.data(), d_rptr, (size_t)(m + 1) * sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(s, cudaStreamSynchronize(st));
    D.on = true;
    return MFS_OK;
}

mfs_status setup_host(mfs_solver* s, int64_t m, int64_t n, int64_t nnz, const int64_t* row, const int64_t* col,
                      const double* val, bool in_order, int64_t ncones, const mfs_cone* cones, HostProblem& P) {
    if (!P.dev.on) build_orders(m, n, nnz, row, col, val, in_order, P);
    // Lorentz cones; unit_end[j] = end of the small cone starting at j, or j+1
    std::vector<int> unit_end(n);
    for (int64_t j = 0; j < n; ++j) unit_end[j] = (int)j + 1;
    int64_t off = 0;
    for (int64_t q = 0; q < ncones; ++q) {
        const int64_t sz = cones[q].size;
        if (cones[q].kind == MFS_CONE_SOC) {
            const int64_t cnnz = (int64_t)P.col_ptr[off + sz] - P.col_ptr[off];
            const bool big = sz > WC || cnnz > WT;
            P.soc_start.push_back((int)off);
            P.soc_size.push_back((int)sz);
            P.soc_big.push_back(big ? 1 : 0);
            if (big)
                P.big_list.push_back((int)P.soc_start.size() - 1);
            else
                unit_end[off] = (int)(off + sz);
        }
        off += sz;
    }
    {
        std::vector<std::pair<int, int>> small;  // small Lorentz cones, in order
        for (size_t q = 0; q < P.soc_start.size(); ++q)
            if (!P.soc_big[q]) small.push_back({P.soc_start[q], P.soc_start[q] + P.soc_size[q]});
        std::vector<mfs::host::ChunkJob> jobs(2);
        jobs[0].ptr = &P.col_ptr;
        jobs[0].nseg = (int)n;
        jobs[0].unit_end = &unit_end;
        jobs[0].out = &P.cc;
        jobs[1].ptr = &P.row_ptr;
        jobs[1].nseg = (int)m;
        jobs[1].unit_end = nullptr;
        jobs[1].out = &P.rc;
        mfs::host::build_chunks(jobs, small, mfs::host::ChunkLimits{WT, WC, PAD});
    }
    if (P.cc.padded >= INT32_MAX - PAD || P.rc.padded >= INT32_MAX - PAD)
        return fail(s, MFS_ERR_INVALID, "too many nonzeros after padding (limit 2^31)");
    // Lorentz cones intersecting each column chunk
    const int ncc = P.cc.count();
    P.cq_lo.resize(ncc);
    P.cq_hi.resize(ncc);
    const int nsoc = (int)P.soc_start.size();
    int lo = 0;
    for (int c = 0; c < ncc; ++c) {
        const int j0 = P.cc.desc[4 * c], j1 = P.cc.desc[4 * c + 1];
        while (lo < nsoc && P.soc_start[lo] + P.soc_size[lo] <= j0) ++lo;
        int hi = lo;
        while (hi < nsoc && P.soc_start[hi] < j1) ++hi;
        P.cq_lo[c] = lo;
        P.cq_hi[c] = hi;
    }
    return MFS_OK;
}

// Padded nonzero arrays: chunk c's nonzeros at desc offset, zero-filled up to a multiple of PAD.
template <typename T, class IdxV, class ValV, class OutI, class OutV>
void pad_chunks(const Chunks& C, const std::vector<int>& ptr, const IdxV& idx, const ValV& val, OutI* pidx,
                OutV* pval) {
    const int nt = mfs::host::threads_for((int64_t)C.padded);
    if (pidx) pidx->resize(C.padded + PAD);
    if (pval) pval->resize(C.padded + PAD);
    // every padded slot is written once: the chunk's nonzeros, then zeros up to the next chunk
    mfs::host::parallel_ranges(C.count(), nt, [&](int64_t lo, int64_t hi, int) {
        for (int64_t c = lo; c < hi; ++c) {
            const int s0 = C.desc[4 * c], s1 = C.desc[4 * c + 1], koff = C.desc[4 * c + 2];
            const int k0 = ptr[s0], k1 = ptr[s1];
            const int end = (c + 1 < C.count()) ? C.desc[4 * (c + 1) + 2] : (int)C.padded + PAD;
            for (int k = k0; k < k1; ++k) {
                if (pidx) (*pidx)[koff + (k - k0)] = idx[k];
                if (pval) (*pval)[koff + (k - k0)] = T(val[k]);
            }
            for (int q = koff + (k1 - k0); q < end; ++q) {
                if (pidx) (*pidx)[q] = 0;
                if (pval) (*pval)[q] = T(0);
            }
        }
    });
    if (C.count() == 0) {
        for (int q = 0; q < (int)C.padded + PAD; ++q) {
            if (pidx) (*pidx)[q] = 0;
            if (pval) (*pval)[q] = T(0);
        }
    }
}

template <typename T>
SweepArgs<T> sweep_args(mfs_solver* s, State<T>& st) {
    SweepArgs<T> a;
    a.col_ptr = s->col_ptr;
    a.cidx = s->cidx;
    a.cval = st.cval;
    a.cdesc = s->cdesc;
    a.cheads = s->cheads;
    a.clong = s->clong;
    a.cq_lo = s->cq_lo;
    a.cq_hi = s->cq_hi;
    a.row_ptr = s->row_ptr;
    a.ridx = s->ridx;
    a.rval = st.rval;
    a.rdesc = s->rdesc;
    a.rheads = s->rheads;
    a.rlong = s->rlong;
    a.soc_start = s->soc_start;
    a.soc_size = s->soc_size;
    a.soc_big = s->soc_big;
    a.big_list = s->big_list;
    a.ctag = s->in_cone;
    a.b = st.b;
    a.c = st.c;
    a.x = st.x;
    a.z = st.z;
    a.del = st.del;
    a.lam = st.lam;
    a.v = st.v;
    a.mu = T(s->set.mu);
    a.ntc = s->ncc;
    a.ntr = s->nrc;
    a.nlc = s->nlc;
    a.nlr = s->nlr;
    a.m = s->m;
    a.n = s->n;
    a.cpad = s->cpad;
    a.rpad = s->rpad;
    return a;
}

template <typename K>
mfs_status persistent_grid(mfs_solver* s, K kernel, int nchunks, int* grid) {
    int per_sm = 0;
    CUDA_TRY(s, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, NT, 0));
    if (per_sm < 1) return fail(s, MFS_ERR_CUDA, "residual kernel does not fit on an SM");
    *grid = std::max(1, std::min((nchunks + NWARP - 1) / NWARP, per_sm * s->num_sms));
    return MFS_OK;
}

template <typename T>
mfs_status residual_grids(mfs_solver* s) {
    int gr = 1, gc = 1;
    TRY(persistent_grid(s, k_row_resid<T>, s->nrc, &gr));
    if (s->has_soc)
        TRY(persistent_grid(s, k_col_resid<T, true>, s->ncc, &gc));
    else
        TRY(persistent_grid(s, k_col_resid<T, false>, s->ncc, &gc));
    s->g_rowres = std::max(s->g_rowres, gr);
    s->g_colres = std::max(s->g_colres, gc);
    return MFS_OK;
}

// ---------------------------------------------------------------------------------- launches

// Staged passes in use (FP32 iterate): on request both; automatically each pass whose layout was
// built on the GPU at no host cost for a large matrix with at least 8 nonzeros per vector entry a
// CTA streams (column pass: o >= 8 m, every CTA streams all of v; row pass: o >= 4 n, every CTA
// streams half of x). On the 10^6 x 2.5*10^6 LP (o = 20 m = 8 n) the staged passes took 105 and
// 94 us against 120 and 110 us for the chunked sweeps.
bool staged_col(const mfs_solver* s) {
    return s->stg_ok && (s->sweep_kind == MFS_SWEEP_STAGED || (s->sweep_kind == MFS_SWEEP_AUTO && s->stg_auto_col));
}
bool staged_row(const mfs_solver* s) {
    return s->stg_ok && (s->sweep_kind == MFS_SWEEP_STAGED || (s->sweep_kind == MFS_SWEEP_AUTO && s->stg_auto_row));
}

inline int warp_grid(int nchunks) {
    return (nchunks + NWARP - 1) / NWARP;
}

// Launch a staged kernel so that it may start while the previous kernel on the stream still runs:
// until it has waited for that kernel (griddepcontrol.wait) it reads only A's staged layout.
template <typename... KArgs, typename... Args>
void launch_dep(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t st, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = MFS_STG_PDL;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);  // an error is left for cudaGetLastError
}

// mid (timing only): recorded after the pass's main kernel, before its combine or long-chunk kernel
template <typename T>
void launch_col(mfs_solver* s, const SweepArgs<T>& a, cudaStream_t st, cudaEvent_t mid = nullptr) {
    if (s->ncc == 0) {
        if (mid) cudaEventRecord(mid, st);
        return;
    }
    if constexpr (std::is_same<T, float>::value) {
        if (staged_col(s)) {
            const StagedArgsT& g = s->stg_col;
            const size_t smem = mfs::staged::smem_bytes(mfs::staged::RB_COL, mfs::staged::S_COL, g.maxg_pad, g.R);
            const int grid = std::min(g.G * g.halves, s->num_sms);
            if (s->has_soc)
                launch_dep(MFS_STAGED_COL_SOC, grid, mfs::staged::NTHREADS, smem, st, g, a);
            else
                launch_dep(MFS_STAGED_COL, grid, mfs::staged::NTHREADS, smem, st, g, a);
            if (mid) cudaEventRecord(mid, st);
            if (g.halves > 1) {
                const int cgrid = (g.nsub + mfs::staged::CWPB - 1) / mfs::staged::CWPB;
                if (s->has_soc)
                    launch_dep(MFS_COL_COMBINE_SOC, cgrid, 32 * mfs::staged::CWPB, 0, st, g, a);
                else
                    launch_dep(MFS_COL_COMBINE, cgrid, 32 * mfs::staged::CWPB, 0, st, g, a);
            }
            return;
        }
    }
    if (s->has_soc) {
        k_col_sweep<T, true><<<warp_grid(s->ncc), NT, 0, st>>>(a);
        if (mid) cudaEventRecord(mid, st);
        if (s->nlc) k_col_long<T, true><<<s->nlc, NT, 0, st>>>(a);
    } else {
        k_col_sweep<T, false><<<warp_grid(s->ncc), NT, 0, st>>>(a);
        if (mid) cudaEventRecord(mid, st);
        if (s->nlc) k_col_long<T, false><<<s->nlc, NT, 0, st>>>(a);
    }
}
template <typename T>
void launch_big(mfs_solver* s, const SweepArgs<T>& a, cudaStream_t st) {
    if constexpr (std::is_same<T, float>::value) {
        if (staged_col(s)) {  // the staged pass's own list
            if (s->stg_nbig) {
                SweepArgs<T> b = a;
                b.big_list = s->stg_big_list;
                k_bigcone_sweep<T><<<s->stg_nbig, NT, 0, st>>>(b);
            }
            return;
        }
    }
    if (s->nbig) k_bigcone_sweep<T><<<s->nbig, NT, 0, st>>>(a);
}
template <typename T, int MODE>
void launch_row_mode(mfs_solver* s, const SweepArgs<T>& a, cudaStream_t st, cudaEvent_t mid = nullptr) {
    if (s->nrc == 0) {
        if (mid) cudaEventRecord(mid, st);
        return;
    }
    if constexpr (std::is_same<T, float>::value && MODE == 0) {
        if (staged_row(s)) {
            const StagedArgsT& g = s->stg_row;
            launch_dep(MFS_STAGED_ROW, std::min(g.G * g.halves, s->num_sms), mfs::staged::NTHREADS,
                       mfs::staged::smem_bytes(mfs::staged::RB_ROW, mfs::staged::S_ROW, g.maxg_pad, g.R), st, g, a);
            if (mid) cudaEventRecord(mid, st);
            if (g.halves > 1)
                launch_dep(mfs::staged::k_row_combine, (int)std::min<int64_t>((s->m + 255) / 256, 8 * s->num_sms), 256,
                           0, st, g, a);
            return;
        }
    }
    k_row_sweep<T, MODE><<<warp_grid(s->nrc), NT, 0, st>>>(a);
    if (mid) cudaEventRecord(mid, st);
    if (s->nlr) k_row_long<T, MODE><<<s->nlr, NT, 0, st>>>(a);
}
template <typename T>
void launch_row(mfs_solver* s, const SweepArgs<T>& a, cudaStream_t st, cudaEvent_t mid = nullptr) {
    launch_row_mode<T, 0>(s, a, st, mid);
}
template <typename T>
void launch_warm_v(mfs_solver* s, const SweepArgs<T>& a, cudaStream_t st) {
    launch_row_mode<T, 1>(s, a, st);
}

template <typename T>
void launch_iteration(mfs_solver* s, const SweepArgs<T>& a, cudaStream_t st) {
    launch_col(s, a, st);
    launch_big(s, a, st);
    launch_row(s, a, st);
}

int launches_per_iteration(const mfs_solver* s) {
    const bool f32 = s->precision == MFS_FP32_MIXED;
    const int col = s->ncc ? ((f32 && staged_col(s)) ? (s->stg_col.halves > 1 ? 2 : 1) : 1 + (s->nlc ? 1 : 0)) : 0;
    const int row = s->nrc ? ((f32 && staged_row(s)) ? (s->stg_row.halves > 1 ? 2 : 1) : 1 + (s->nlr ? 1 : 0)) : 0;
    const int big = (f32 && staged_col(s)) ? (s->stg_nbig ? 1 : 0) : (s->nbig ? 1 : 0);
    return col + big + row;
}

template <typename T>
mfs_status run_iters(mfs_solver* s, State<T>& st, int64_t k) {
    if (k <= 0) return MFS_OK;
    SweepArgs<T> a = sweep_args(s, st);
    const int K = std::max(1, (int)s->set.check_every);
    if (k >= K) {
        if (!st.graph || st.graph_iters != K) {
            if (st.graph) {
                cudaGraphExecDestroy(st.graph);
                st.graph = nullptr;
            }
            cudaGraph_t g = nullptr;
            CUDA_TRY(s, cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal));
            for (int i = 0; i < K; ++i) launch_iteration(s, a, s->cap);
            CUDA_TRY(s, cudaStreamEndCapture(s->cap, &g));
            cudaError_t e = cudaGraphInstantiate(&st.graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                st.graph = nullptr;
                return fail(s, MFS_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
            }
            st.graph_iters = K;
        }
        while (k >= K) {
            CUDA_TRY(s, cudaGraphLaunch(st.graph, s->stream));
            k -= K;
            s->iter += K;
        }
    }
    for (int64_t i = 0; i < k; ++i) launch_iteration(s, a, s->stream);
    s->iter += k;
    CUDA_TRY(s, cudaGetLastError());
    return MFS_OK;
}

double stop_measure(const mfs_residuals_t& r, int rule) {
    return rule == MFS_STOP_SCS_L2 ? r.r_scs : rule == MFS_STOP_OSQP_INF ? r.r_osqp : r.kkt;
}

template <typename T>
mfs_status residuals_t(mfs_solver* s, State<T>& st, mfs_residuals_t* out, bool write_all_s) {
    SweepArgs<T> a = sweep_args(s, st);
    ResidArgs r;
    r.part_row = s->part_row;
    r.part_col = s->part_col;
    r.part_big = s->part_big;
    r.s_buf = s->s_buf;
    r.r_buf = s->r_buf;
    r.write_all_s = write_all_s ? 1 : 0;
    const int gr = s->nrc ? s->g_rowres : 0, gc = s->ncc ? s->g_colres : 0;
    if (gr) k_row_resid<T><<<gr, NT, 0, s->stream>>>(a, r);
    if (gc) {
        if (s->has_soc)
            k_col_resid<T, true><<<gc, NT, 0, s->stream>>>(a, r);
        else
            k_col_resid<T, false><<<gc, NT, 0, s->stream>>>(a, r);
    }
    if (s->nbig) k_bigcone_resid<T><<<s->nbig, NT, 0, s->stream>>>(a, r, s->nbig);
    k_resid_finalize<<<1, 32 * NFALL, 0, s->stream>>>(s->part_row, gr, s->part_col, gc, s->part_big, s->nbig,
                                                      s->status);
    CUDA_TRY(s, cudaGetLastError());
    if (out) {
        CUDA_TRY(s, cudaMemcpyAsync(s->h_status, s->status, NSTATUS * sizeof(double), cudaMemcpyDeviceToHost,
                                    s->stream));
        if (s->stg_ok) CUDA_TRY(s, cudaMemcpyAsync(s->h_err, s->stg_err, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
        CUDA_TRY(s, cudaStreamSynchronize(s->stream));
        if (s->stg_ok && *s->h_err)
            return fail(s, MFS_ERR_TIMEOUT, "a staged sweep gave up waiting for a block of its vector");
        const double* h = s->h_status;
        out->r_prim = h[S_RPRIM];
        out->r_dual = h[S_RDUAL];
        out->r_cone = h[S_RCONE];
        out->r_gap = h[S_RGAP];
        out->kkt = h[S_KKT];
        out->pobj = h[S_POBJ];
        out->dobj = h[S_DOBJ];
        out->nrm_res_p = h[S_NRES];
        out->nrm_b = h[S_NB];
        out->nrm_xdist = h[S_NXDIST];
        out->nrm_x = h[S_NX];
        out->nrm_sdist = h[S_NSDIST];
        out->nrm_c = h[S_NC];
        out->nrm_atl_c = h[S_NATLC];
        out->inf_res_p = h[S_IRES];
        out->inf_ax = h[S_IAX];
        out->inf_b = h[S_IB];
        out->inf_atl_c = h[S_IATLC];
        out->inf_atl = h[S_IATL];
        out->inf_c = h[S_IC];
        out->inf_x = h[S_IX];
        out->inf_xdist = h[S_IXDIST];
        out->inf_sdist = h[S_ISDIST];
        mfs::stop_measures(out, s->set.osqp_rel);
        out->iter = s->iter;
    }
    return MFS_OK;
}

template <typename D, typename S>
void convert(D* dst, const S* src, int64_t count, cudaStream_t st) {
    if (count <= 0) return;
    const int blocks = (int)std::min<int64_t>((count + 255) / 256, 148 * 16);
    k_convert<D, S><<<blocks, 256, 0, st>>>(dst, src, (long long)count);
}

// Warm start from FP64 device vectors (x, lam required; z, del nullable).
template <typename T>
mfs_status warm_start_t(mfs_solver* s, State<T>& st, const double* x, const double* lam, const double* z,
                        const double* del) {
    convert(st.x, x, s->n, s->stream);
    convert(st.lam, lam, s->m, s->stream);
    const int pb = 256;
    if (z) {
        convert(st.z, z, s->n, s->stream);
    } else if (s->n) {
        k_proj_orthant<T><<<(int)std::min<int64_t>((s->n + pb - 1) / pb, 148 * 16), pb, 0, s->stream>>>(st.z, x, s->n);
        if (s->nsoc) k_proj_soc<T><<<(s->nsoc + pb - 1) / pb, pb, 0, s->stream>>>(st.z, x, s->soc_start, s->soc_size, s->nsoc);
    }
    if (del) {
        convert(st.del, del, s->n, s->stream);
    } else {
        // s_buf = c + A^T lambda (FP64 accumulation), then delta = proj_K(s_buf)
        TRY(residuals_t(s, st, nullptr, true));
        if (s->n) {
            k_proj_orthant<T><<<(int)std::min<int64_t>((s->n + pb - 1) / pb, 148 * 16), pb, 0, s->stream>>>(
                st.del, s->s_buf, s->n);
            if (s->nsoc)
                k_proj_soc<T><<<(s->nsoc + pb - 1) / pb, pb, 0, s->stream>>>(st.del, s->s_buf, s->soc_start,
                                                                             s->soc_size, s->nsoc);
        }
    }
    // v = F_U (b - A x) - lambda/mu
    launch_warm_v(s, sweep_args(s, st), s->stream);
    CUDA_TRY(s, cudaGetLastError());
    CUDA_TRY(s, cudaStreamSynchronize(s->stream));
    s->iter = 0;
    return MFS_OK;
}

// Padded column (col = true) or row arrays filled on the device from the orders of device_orders:
// indices into *pidx and/or values (as T) into *pval, zero in the padding (as pad_chunks writes).
template <typename T>
mfs_status pad_on_device(mfs_solver* s, const HostProblem& P, bool col, int** pidx, T** pval) {
    const Chunks& C = col ? P.cc : P.rc;
    const size_t len = (size_t)C.padded + PAD;
    if (pidx) {
        TRY(dalloc(s, pidx, len));
        CUDA_TRY(s, cudaMemsetAsync(*pidx, 0, len * sizeof(int), s->stream));
    }
    if (pval) {
        TRY(dalloc(s, pval, len));
        CUDA_TRY(s, cudaMemsetAsync(*pval, 0, len * sizeof(T), s->stream));
    }
    const int nch = C.count();
    if (nch > 0)
        mfs::setup::k_pad<T><<<(int)std::min<int64_t>((nch + 7) / 8, 8 * s->num_sms), 256, 0, s->stream>>>(
            col ? s->cdesc : s->rdesc, nch, col ? s->col_ptr : s->row_ptr, col ? P.dev.crow : P.dev.rcol,
            col ? P.dev.cval : P.dev.rval, pidx ? *pidx : nullptr, pval ? *pval : nullptr);
    CUDA_TRY(s, cudaGetLastError());
    return MFS_OK;
}

// b and c are host arrays, or device arrays when bc_on_device
template <typename T>
mfs_status alloc_state(mfs_solver* s, State<T>& st, const HostProblem& P, const double* b, const double* c,
                       bool bc_on_device) {
    // x and v, the vectors the staged sweeps copy in whole blocks, are padded to a multiple of the block
    const int64_t npad = (int64_t)(s->n + mfs::staged::RB_ROW - 1) / mfs::staged::RB_ROW * mfs::staged::RB_ROW;
    const int64_t mpad = (int64_t)(s->m + mfs::staged::RB_COL - 1) / mfs::staged::RB_COL * mfs::staged::RB_COL;
    TRY(dalloc(s, &st.x, npad));
    TRY(dalloc(s, &st.z, s->n));
    TRY(dalloc(s, &st.del, s->n));
    TRY(dalloc(s, &st.lam, s->m));
    TRY(dalloc(s, &st.v, mpad));
    if (bc_on_device) {
        TRY(dalloc(s, &st.b, s->m));
        TRY(dalloc(s, &st.c, s->n));
        convert(st.b, b, s->m, s->stream);
        convert(st.c, c, s->n, s->stream);
        CUDA_TRY(s, cudaGetLastError());
    } else {
        std::vector<T> hb(b, b + s->m), hc(c, c + s->n);
        TRY(upload(s, &st.b, hb.data(), hb.size()));
        TRY(upload(s, &st.c, hc.data(), hc.size()));
    }
    if (P.dev.on) {
        TRY(pad_on_device<T>(s, P, true, nullptr, &st.cval));
        TRY(pad_on_device<T>(s, P, false, nullptr, &st.rval));
    } else {
        mfs::host::uvec<T> pval;
        pad_chunks<T>(P.cc, P.col_ptr, P.csc_row, P.csc_val, (mfs::host::uvec<int>*)nullptr, &pval);
        TRY(upload(s, &st.cval, pval.data(), pval.size()));
        pad_chunks<T>(P.rc, P.row_ptr, P.csr_col, P.csr_val, (mfs::host::uvec<int>*)nullptr, &pval);
        TRY(upload(s, &st.rval, pval.data(), pval.size()));
    }
    CUDA_TRY(s, cudaMemsetAsync(st.x, 0, sizeof(T) * std::max<int64_t>(npad, 1), s->stream));
    CUDA_TRY(s, cudaMemsetAsync(st.z, 0, sizeof(T) * std::max(s->n, 1), s->stream));
    CUDA_TRY(s, cudaMemsetAsync(st.del, 0, sizeof(T) * std::max(s->n, 1), s->stream));
    CUDA_TRY(s, cudaMemsetAsync(st.lam, 0, sizeof(T) * std::max(s->m, 1), s->stream));
    CUDA_TRY(s, cudaMemsetAsync(st.v, 0, sizeof(T) * std::max<int64_t>(mpad, 1), s->stream));
    return MFS_OK;
}

// Staged sweeps for an FP32 problem with orthant cones only: both layouts, the row norms, the
// kernels' shared-memory limits; the automatic choice takes a staged pass when the matrix is large
// and the gathered vector small against its nonzeros (every CTA reads the whole vector).
// The staged layout of one pass built on the GPU (mfs_setup.cuh) from a device order (segment
// pointers, gathered indices, FP64 values), for the plan S (groups and warp segments) made on the
// host: the entries split by block, the warp ranges, the lane layout with its overflow slots and
// fold lists. *ok is false (and nothing kept) when a group's sums and overflow sums would not fit
// in shared memory (smem_limit) or in the 16-bit slot field.
mfs_status staged_on_device(mfs_solver* s, const StagedHost& S, const int* d_ptr, int nseg, int64_t o,
                            const int* d_idx, const double* d_val, int rb, int stages, size_t smem_limit,
                            mfs::staged::StagedArgs& g, bool* ok) {
    namespace su = mfs::setup;
    using mfs::staged::NW;
    *ok = false;
    const int G = S.G, R = S.R, NW1 = NW + 1;
    const int64_t nb = (int64_t)G * R, nr = nb * NW;
    cudaStream_t st = s->stream;
    const int grid = 8 * s->num_sms;
    std::vector<void*> tmp;
    struct Free {
        std::vector<void*>& v;
        ~Free() {
            for (void* q : v) cudaFree(q);
        }
    } release{tmp};
    auto grab = [&](void** q, size_t bytes) -> mfs_status {
        cudaError_t e = mfs::device_malloc(q, std::max<size_t>(bytes, 16));
        if (e != cudaSuccess)
            return fail(s, e == cudaErrorMemoryAllocation ? MFS_ERR_OOM : MFS_ERR_CUDA,
                        std::string("cudaMalloc: ") + cudaGetErrorString(e));
        tmp.push_back(*q);
        return MFS_OK;
    };
    int *grp = nullptr, *wseg = nullptr, *split = nullptr, *wovf = nullptr, *fold_ptr = nullptr;
    TRY(upload(s, &grp, S.grp.data(), S.grp.size()));
    TRY(upload(s, &wseg, S.wseg.data(), S.wseg.size()));
    TRY(dalloc(s, &split, (size_t)nb * NW1));
    TRY(dalloc(s, &wovf, (size_t)G * NW1));
    TRY(dalloc(s, &fold_ptr, (size_t)G * NW + 1));
    int *segof = nullptr, *cnt = nullptr, *bstart = nullptr, *npieces = nullptr, *ovf = nullptr, *c1 = nullptr,
        *c2 = nullptr, *s1 = nullptr, *s2 = nullptr, *slots_max = nullptr;
    int2 *ent = nullptr, *lent = nullptr;
    const size_t ns1 = (size_t)nseg + 1;
    TRY(grab((void**)&segof, (size_t)o * sizeof(int)));
    TRY(grab((void**)&cnt, (size_t)nb * sizeof(int)));
    TRY(grab((void**)&bstart, (size_t)nb * sizeof(int)));
    TRY(grab((void**)&ent, (size_t)o * sizeof(int2)));
    TRY(grab((void**)&npieces, ns1 * sizeof(int)));
    TRY(grab((void**)&ovf, ns1 * sizeof(int)));
    TRY(grab((void**)&c1, ns1 * sizeof(int)));
    TRY(grab((void**)&c2, ns1 * sizeof(int)));
    TRY(grab((void**)&s1, ns1 * sizeof(int)));
    TRY(grab((void**)&s2, ns1 * sizeof(int)));
    TRY(grab((void**)&slots_max, sizeof(int)));
    TRY(dalloc(s, &lent, (size_t)std::max<int64_t>(o, 1)));
    su::k_seg_of<<<grid, 256, 0, st>>>(d_ptr, nseg, segof);
    su::k_stg_count<<<G, 256, (size_t)R * sizeof(int), st>>>(d_ptr, grp, d_idx, R, rb, cnt);
    TRY(device_scan(s, cnt, bstart, nb, nullptr));
    const size_t scat_smem = (size_t)(1 + su::SNT / 32) * R * sizeof(int);
    CUDA_TRY(s, cudaFuncSetAttribute(su::k_stg_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)scat_smem));
    su::k_stg_scatter<<<G, su::SNT, scat_smem, st>>>(d_ptr, grp, segof, d_idx, d_val, R, rb, bstart, ent);
    su::k_stg_split<<<(int)std::min<int64_t>((nb + 255) / 256, grid), 256, 0, st>>>(ent, bstart, cnt, wseg, R, (int)nb,
                                                                                   NW1, split);
    CUDA_TRY(s, cudaMemsetAsync(npieces, 0, ns1 * sizeof(int), st));
    CUDA_TRY(s, cudaMemsetAsync(slots_max, 0, sizeof(int), st));
    const int lgrid = (int)std::min<int64_t>((nr + 127) / 128, 64 * s->num_sms);
    su::k_stg_lanes<0><<<lgrid, 128, 0, st>>>(ent, split, nr, NW1, R, grp, npieces, nullptr, nullptr);
    // overflow slots and fold lists from two device-wide scans
    su::k_stg_ovf_counts<<<grid, 256, 0, st>>>(npieces, nseg, c1, c2);
    int tot1 = 0, nfold = 0;
    TRY(device_scan(s, c1, s1, nseg, &tot1));
    TRY(device_scan(s, c2, s2, nseg, &nfold));
    CUDA_TRY(s, cudaMemcpyAsync(s1 + nseg, &tot1, sizeof(int), cudaMemcpyHostToDevice, st));
    CUDA_TRY(s, cudaMemcpyAsync(s2 + nseg, &nfold, sizeof(int), cudaMemcpyHostToDevice, st));
    int2* fold = nullptr;
    TRY(dalloc(s, &fold, (size_t)std::max(nfold, 1)));
    su::k_stg_ovf_place<<<grid, 256, 0, st>>>(grp, G, npieces, s1, s2, nseg, ovf, fold);
    su::k_stg_ovf_warps<<<(G * NW1 + 255) / 256, 256, 0, st>>>(grp, G, wseg, NW1, s1, s2, nseg, wovf, fold_ptr,
                                                                slots_max);
    su::k_stg_lanes<1><<<lgrid, 128, 0, st>>>(ent, split, nr, NW1, R, grp, nullptr, ovf, lent);
    int hmax = 0;
    CUDA_TRY(s, cudaMemcpyAsync(&hmax, slots_max, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(s, cudaGetLastError());
    CUDA_TRY(s, cudaStreamSynchronize(st));
    const int slots = (hmax + 3) / 4 * 4;
    if (slots >= mfs::staged::MAXSLOT || mfs::staged::smem_bytes(rb, stages, slots, R) > smem_limit) return MFS_OK;
    g.ent = lent;
    g.split = split;
    g.grp = grp;
    g.wseg = wseg;
    g.wovf = wovf;
    g.fold_ptr = fold_ptr;
    g.fold = fold;
    g.nent = (int)o;
    g.maxg_pad = slots;
    *ok = true;
    return MFS_OK;
}

// Whether a staged pass split into `groups` groups can keep them whole: the average group (segments
// per group) must fit in the shared memory that plan_staged leaves for the sums (a quick test before
// planning; plan_staged decides).
bool groups_may_fit(int nseg, int nother, int groups, int rb, int stages, size_t smem_limit) {
    const int R = std::max(1, (nother + rb - 1) / rb);
    const size_t fixed = mfs::staged::smem_bytes(rb, stages, 0, R);
    if (fixed + 4096 * 4 > smem_limit) return false;
    const size_t maxg = std::min<size_t>(mfs::staged::MAXG, (smem_limit - fixed) / 16 * 4);
    return (size_t)((nseg + groups - 1) / groups) <= maxg;
}

// The staged passes access the iterate's vectors evict-last. Such lines stay in L2 only within the
// context's persisting set-aside; with settings.l2_keep the first staged solver of a device raises it
// to the device's maximum and the last one to be destroyed puts the previous value back (where it
// cannot be raised the hint stays a hint). The set-aside is L2 that other work in the context does
// not get while it is raised.
std::mutex g_keep_mu;
struct KeepRef {
    int count = 0;
    size_t prev = 0;
};
KeepRef g_keep[64];

void keep_acquire(mfs_solver* s) {
    if (s->device < 0 || s->device >= 64) return;
    std::lock_guard<std::mutex> lk(g_keep_mu);
    KeepRef& k = g_keep[s->device];
    if (k.count == 0) {
        int maxp = 0;
        size_t cur = 0;
        if (cudaDeviceGetAttribute(&maxp, cudaDevAttrMaxPersistingL2CacheSize, s->device) != cudaSuccess ||
            cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize) != cudaSuccess) {
            (void)cudaGetLastError();
            return;
        }
        k.prev = cur;
        if (cur < (size_t)maxp && cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, (size_t)maxp) != cudaSuccess)
            (void)cudaGetLastError();
    }
    ++k.count;
    s->keep_l2 = true;
}

void keep_release(mfs_solver* s) {
    if (!s->keep_l2) return;
    s->keep_l2 = false;
    std::lock_guard<std::mutex> lk(g_keep_mu);
    KeepRef& k = g_keep[s->device];
    if (--k.count == 0 && cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, k.prev) != cudaSuccess)
        (void)cudaGetLastError();
}

mfs_status setup_staged(mfs_solver* s, const HostProblem& P) {
    using namespace mfs::staged;
    int optin = 0;
    CUDA_TRY(s, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, s->device));
    StagedHost C, W;
    // small Lorentz cones stay within one warp's columns (its epilogue projects them)
    std::vector<int> unit_start;
    if (s->has_soc) {
        unit_start.resize(P.n);
        for (int j = 0; j < P.n; ++j) unit_start[j] = j;
        for (size_t q = 0; q < P.soc_start.size(); ++q)
            if (P.soc_size[q] <= WC)
                for (int t = 1; t < P.soc_size[q]; ++t) unit_start[P.soc_start[q] + t] = P.soc_start[q];
    }
    // The column pass likewise, in parts where v is long enough (each CTA streams at least 8 blocks)
    // and the column groups of half as many CTAs still fit; k_col_combine then adds the parts and
    // runs the epilogue, each warp of the split on its own warp range held in shared memory.
    int col_parts = 1;
    {
        const int R = std::max(1, (P.m + RB_COL - 1) / RB_COL);
        bool ok = false;
        for (int h = COL_PARTS_MAX; h >= 1 && !ok; h /= 2) {
            const int groups = std::max(1, s->num_sms / h);
            if (h > 1 && (R / h < 8 || !groups_may_fit(P.n, P.m, groups, RB_COL, S_COL, (size_t)optin))) continue;
            StagedHost T;
            if (!plan_staged(P.col_ptr, P.n, P.m, groups, RB_COL, S_COL, (size_t)optin, T,
                             s->has_soc ? &unit_start : nullptr))
                continue;
            if (h > 1 && T.G > groups) continue;  // groups split for shared memory: fewer parts
            C = std::move(T);
            col_parts = h;
            ok = true;
        }
        if (!ok) return MFS_OK;  // vectors too long for the split tables: chunked sweeps only
    }
    // The row pass splits each row group over `row_parts` CTAs, each streaming its share of x's
    // blocks into partial row sums (k_row_combine adds them). Two parts, or more where every CTA
    // still streams at least 8 blocks and the larger row groups still fit in shared memory.
    int row_parts = ROW_HALVES;
    {
        const int R = std::max(1, (P.n + RB_ROW - 1) / RB_ROW);
        bool ok = false;
        for (int h = ROW_PARTS_MAX; h >= ROW_HALVES && !ok; h /= 2) {
            const int groups = std::max(1, s->num_sms / h);
            if (h > ROW_HALVES && (R / h < 8 || !groups_may_fit(P.m, P.n, groups, RB_ROW, S_ROW, (size_t)optin)))
                continue;
            StagedHost T;
            if (!plan_staged(P.row_ptr, P.m, P.n, groups, RB_ROW, S_ROW, (size_t)optin, T)) continue;
            if (h > ROW_HALVES && T.G > groups) continue;  // groups split for shared memory: fewer parts
            W = std::move(T);
            row_parts = h;
            ok = true;
        }
        if (!ok) return MFS_OK;
    }
    // the orders on the device: where the host built them, uploaded for the set-up only
    const bool dev = P.dev.on;
    const int *crow = P.dev.crow, *rcol = P.dev.rcol;
    const double *cval = P.dev.cval, *rval = P.dev.rval;
    std::vector<void*> tmp;
    struct Free {
        std::vector<void*>& v;
        ~Free() {
            for (void* q : v) cudaFree(q);
        }
    } release{tmp};
    if (!dev) {
        auto up = [&](const void* src, size_t bytes, const void** dst) -> mfs_status {
            void* q = nullptr;
            cudaError_t e = mfs::device_malloc(&q, std::max<size_t>(bytes, 16));
            if (e != cudaSuccess)
                return fail(s, e == cudaErrorMemoryAllocation ? MFS_ERR_OOM : MFS_ERR_CUDA,
                            std::string("cudaMalloc: ") + cudaGetErrorString(e));
            tmp.push_back(q);
            if (bytes) CUDA_TRY(s, cudaMemcpyAsync(q, src, bytes, cudaMemcpyHostToDevice, s->stream));
            *dst = q;
            return MFS_OK;
        };
        TRY(up(P.csc_row.data(), (size_t)P.o * sizeof(int), (const void**)&crow));
        TRY(up(P.csc_val.data(), (size_t)P.o * sizeof(double), (const void**)&cval));
        TRY(up(P.csr_col.data(), (size_t)P.o * sizeof(int), (const void**)&rcol));
        TRY(up(P.csr_val.data(), (size_t)P.o * sizeof(double), (const void**)&rval));
    }
    StagedArgs gc{}, gr{};
    bool okc = false, okr = false;
    TRY(staged_on_device(s, C, s->col_ptr, P.n, P.o, crow, cval, RB_COL, S_COL, (size_t)optin, gc, &okc));
    if (!okc) return MFS_OK;
    TRY(staged_on_device(s, W, s->row_ptr, P.m, P.o, rcol, rval, RB_ROW, S_ROW, (size_t)optin, gr, &okr));
    if (!okr) return MFS_OK;
    TRY(dalloc(s, &s->stg_err, 1));
    CUDA_TRY(s, cudaMemsetAsync(s->stg_err, 0, sizeof(int), s->stream));
    CUDA_TRY(s, cudaMallocHost(&s->h_err, sizeof(int)));
    *s->h_err = 0;
    auto fill = [&](const StagedHost& H, StagedArgs& g, const float* vec, int halves, int nseg) -> mfs_status {
        g.vec = vec;
        g.err = s->stg_err;
        g.G = H.G;
        g.R = H.R;
        g.halves = halves;
        g.nseg = nseg;
        g.part = nullptr;
        if (halves > 1) TRY(dalloc(s, &g.part, (size_t)halves * std::max(nseg, 1)));
        g.spin = 1 << 24;
        g.no_loads = 0;
        return MFS_OK;
    };
    gc.wcone = nullptr;
    gc.ctag = nullptr;
    gc.soc_big = nullptr;
    if (s->has_soc) {  // each warp's Lorentz cones: those starting within its columns
        std::vector<int2> wc((size_t)C.G * NW);
        for (int g2 = 0; g2 < C.G; ++g2)
            for (int w = 0; w < NW; ++w) {
                const int c0 = C.grp[g2] + C.wseg[(size_t)g2 * (NW + 1) + w];
                const int c1 = C.grp[g2] + C.wseg[(size_t)g2 * (NW + 1) + w + 1];
                const int q0 = (int)(std::lower_bound(P.soc_start.begin(), P.soc_start.end(), c0) - P.soc_start.begin());
                const int q1 = (int)(std::lower_bound(P.soc_start.begin(), P.soc_start.end(), c1) - P.soc_start.begin());
                wc[(size_t)g2 * NW + w] = make_int2(q0, q1);
            }
        int2* d_wc = nullptr;
        TRY(upload(s, &d_wc, wc.data(), wc.size()));
        gc.wcone = d_wc;
        // the staged pass fuses every cone of at most WC columns, however many nonzeros it has (the
        // chunked sweeps leave cones with more than WT nonzeros to the big-cone kernel as well)
        std::vector<unsigned char> tag((size_t)P.n, 0), big(P.soc_start.size(), 0);
        std::vector<int> blist;
        for (size_t q = 0; q < P.soc_start.size(); ++q) {
            big[q] = P.soc_size[q] > WC ? 1 : 0;
            if (big[q]) blist.push_back((int)q);
            for (int t = 0; t < P.soc_size[q]; ++t) tag[(size_t)P.soc_start[q] + t] = big[q] ? 2 : 1;
        }
        unsigned char *d_tag = nullptr, *d_big = nullptr;
        TRY(upload(s, &d_tag, tag.data(), tag.size()));
        TRY(upload(s, &d_big, big.data(), big.size()));
        if (!blist.empty()) TRY(upload(s, &s->stg_big_list, blist.data(), blist.size()));
        s->stg_nbig = (int)blist.size();
        gc.ctag = d_tag;
        gc.soc_big = d_big;
    }
    s->stg_col = gc;
    s->stg_row = gr;
    TRY(fill(C, s->stg_col, s->s32.v, col_parts, P.n));
    s->stg_col.csub = nullptr;
    s->stg_col.nsub = 0;
    if (col_parts > 1) {
        // k_col_combine's pieces: about CSUB columns, a cut inside a fused cone moved to its end
        std::vector<int4> sub;
        size_t q = 0;  // the next Lorentz cone
        for (int c0 = 0; c0 < P.n;) {
            int c1 = std::min(P.n, c0 + mfs::staged::CSUB);
            if (s->has_soc && c1 < P.n && unit_start[c1] != c1) {
                const int st = unit_start[c1];
                const size_t k = (size_t)(std::lower_bound(P.soc_start.begin(), P.soc_start.end(), st) -
                                          P.soc_start.begin());
                c1 = st + P.soc_size[k];
            }
            const size_t q0 = q;
            while (q < P.soc_start.size() && P.soc_start[q] < c1) ++q;
            sub.push_back(make_int4(c0, c1, (int)q0, (int)q));
            c0 = c1;
        }
        int4* d_sub = nullptr;
        TRY(upload(s, &d_sub, sub.data(), sub.size()));
        s->stg_col.csub = d_sub;
        s->stg_col.nsub = (int)sub.size();
    }
    TRY(fill(W, s->stg_row, s->s32.x, row_parts, P.m));
    float *d_rinv = nullptr, *d_dinv = nullptr;
    TRY(dalloc(s, &d_rinv, (size_t)std::max(P.m, 1)));
    TRY(dalloc(s, &d_dinv, (size_t)std::max(P.n, 1)));
    if (P.m > 0)
        mfs::setup::k_row_inv<<<(int)std::min<int64_t>((P.m + 255) / 256, 8 * s->num_sms), 256, 0, s->stream>>>(
            s->row_ptr, rval, P.m, d_rinv);
    if (P.n > 0)
        mfs::setup::k_col_inv<<<(int)std::min<int64_t>((P.n + 255) / 256, 8 * s->num_sms), 256, 0, s->stream>>>(
            s->col_ptr, P.n, d_dinv);
    CUDA_TRY(s, cudaGetLastError());
    CUDA_TRY(s, cudaStreamSynchronize(s->stream));  // the uploaded orders are freed on return
    s->stg_row.rinv = d_rinv;
    s->stg_col.dinv = d_dinv;
    // the limit is a property of the kernel, shared by all solvers: allow the device's maximum
    CUDA_TRY(s, cudaFuncSetAttribute(MFS_STAGED_COL, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    CUDA_TRY(s, cudaFuncSetAttribute(MFS_STAGED_COL_SOC, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    CUDA_TRY(s, cudaFuncSetAttribute(MFS_STAGED_ROW, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    s->stg_ok = true;
#if MFS_STG_KEEP
    if (s->set.l2_keep) keep_acquire(s);
#endif
    return MFS_OK;
}


template <typename D, typename S>
void copy_state(mfs_solver* s, State<D>& dst, State<S>& src) {
    convert(dst.x, src.x, s->n, s->stream);
    convert(dst.z, src.z, s->n, s->stream);
    convert(dst.del, src.del, s->n, s->stream);
    convert(dst.lam, src.lam, s->m, s->stream);
    convert(dst.v, src.v, s->m, s->stream);
}

int64_t bytes_per_iter(const mfs_solver* s, int precision) {
    const int64_t o = s->o, n = s->n, m = s->m;
    return precision == MFS_FP64 ? 24 * o + 68 * n + 44 * m : 16 * o + 36 * n + 24 * m;
}

bool finite_all(const double* p, int64_t count) {
    for (int64_t i = 0; i < count; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

void destroy_graphs(mfs_solver* s) {
    if (s->s32.graph) cudaGraphExecDestroy(s->s32.graph);
    if (s->s64.graph) cudaGraphExecDestroy(s->s64.graph);
    s->s32.graph = nullptr;
    s->s64.graph = nullptr;
}

}  // namespace

template <typename T>
static mfs_status get_solution_t(mfs_solver* s, State<T>& st, double* x, double* lam, double* z, double* del,
                                 bool host) {
    double* tmp = nullptr;
    const int64_t n = s->n, m = s->m;
    if (host) {
        cudaError_t e = cudaMallocAsync((void**)&tmp, std::max<int64_t>(3 * n + m, 1) * sizeof(double), s->stream);
        if (e != cudaSuccess) return fail(s, MFS_ERR_OOM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
    }
    double* dst[4] = {x, lam, z, del};
    const T* src[4] = {st.x, st.lam, st.z, st.del};
    const int64_t cnt[4] = {n, m, n, n};
    int64_t off = 0;
    std::vector<HostCopy> down;
    for (int q = 0; q < 4; ++q) {
        if (!dst[q] || !cnt[q]) continue;
        double* d = host ? tmp + off : dst[q];
        convert(d, src[q], cnt[q], s->stream);
        if (host) down.push_back({dst[q], d, (size_t)cnt[q] * sizeof(double)});
        off += cnt[q];
    }
    CUDA_TRY(s, cudaGetLastError());
    mfs_status r = MFS_OK;
    if (host) r = download_pinned(s, down, s->stream);
    if (tmp) cudaFreeAsync(tmp, s->stream);
    CUDA_TRY(s, cudaGetLastError());
    CUDA_TRY(s, cudaStreamSynchronize(s->stream));
    return r;
}

template <typename T>
static mfs_status time_kernels_t(mfs_solver* s, State<T>& st, int64_t k, double* out, bool split) {
    // k iterations back to back, an event after each kernel group (a pass's main kernel, its
    // combine or long-chunk kernel, the big cones, ...); one wait at the end, so that no host round
    // trip idles the GPU between iterations. out: column main, column rest, big cones, row main,
    // row rest, whole iteration (average milliseconds). Without `split` the events fall only between
    // passes (a pass's kernels keep their programmatic overlap; its time is in "main").
    SweepArgs<T> a = sweep_args(s, st);
    const int64_t kk = std::max<int64_t>(k, 0);
    const int E = split ? 5 : 3;  // events per iteration
    std::vector<cudaEvent_t> ev((size_t)(E * kk + 1), nullptr);
    mfs_status r = MFS_OK;
    for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            e = nullptr;
            r = fail(s, MFS_ERR_CUDA, "cudaEventCreate failed");
            break;
        }
    double t[5] = {0, 0, 0, 0, 0}, tall = 0;
    if (r == MFS_OK) {
        cudaEventRecord(ev[0], s->stream);
        for (int64_t i = 0; i < kk; ++i) {
            cudaEvent_t* e = ev.data() + E * i;
            if (split) {
                launch_col(s, a, s->stream, e[1]);
                cudaEventRecord(e[2], s->stream);
                launch_big(s, a, s->stream);
                cudaEventRecord(e[3], s->stream);
                launch_row(s, a, s->stream, e[4]);
                cudaEventRecord(e[5], s->stream);
            } else {
                launch_col(s, a, s->stream);
                cudaEventRecord(e[1], s->stream);
                launch_big(s, a, s->stream);
                cudaEventRecord(e[2], s->stream);
                launch_row(s, a, s->stream);
                cudaEventRecord(e[3], s->stream);
            }
        }
        cudaError_t e = cudaEventSynchronize(ev[E * kk]);
        if (e != cudaSuccess) r = fail(s, MFS_ERR_CUDA, std::string("time_kernels: ") + cudaGetErrorString(e));
        for (int64_t i = 0; i < kk && r == MFS_OK; ++i)
            for (int q = 0; q < E; ++q) {
                float ms = 0;
                cudaEventElapsedTime(&ms, ev[E * i + q], ev[E * i + q + 1]);
                t[q] += ms;
            }
        if (kk > 0 && r == MFS_OK) {
            float ms = 0;
            cudaEventElapsedTime(&ms, ev[0], ev[E * kk]);
            tall = ms;
        }
    }
    for (auto& e : ev)
        if (e) cudaEventDestroy(e);
    if (r != MFS_OK) return r;
    s->iter += k;
    const double kd = kk > 0 ? (double)kk : 1.0;
    if (split) {
        out[0] = t[0] / kd;  // column main kernel
        out[1] = t[1] / kd;  // column combine / long chunks
        out[2] = t[2] / kd;  // big cones
        out[3] = t[3] / kd;  // row main kernel
        out[4] = t[4] / kd;  // row combine / long chunks
    } else {  // per pass: column, big cones, row
        out[0] = t[0] / kd;
        out[1] = 0.0;
        out[2] = t[1] / kd;
        out[3] = t[2] / kd;
        out[4] = 0.0;
    }
    out[5] = tall / kd;
    CUDA_TRY(s, cudaGetLastError());
    return MFS_OK;
}

static void literal_free(mfs_solver* s);

static mfs_status warm_start_impl(mfs_solver* s, const double* x, const double* lam, const double* z,
                                  const double* del, bool host) {
    if (!s) return MFS_ERR_INVALID;
    literal_free(s);
    if ((s->n && !x) || (s->m && !lam)) return fail(s, MFS_ERR_INVALID, "x and lambda are required");
    CUDA_TRY(s, cudaSetDevice(s->device));
    const double *dx = x, *dl = lam, *dz = z, *dd = del;
    double* tmp = nullptr;
    if (host) {
        const int64_t need = 3 * (int64_t)s->n + s->m;
        cudaError_t e = cudaMallocAsync((void**)&tmp, std::max<int64_t>(need, 1) * sizeof(double), s->stream);
        if (e != cudaSuccess) return fail(s, MFS_ERR_OOM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
        double* p = tmp;
        auto put = [&](const double* h, int64_t cnt, const double*& d) -> cudaError_t {
            if (!h) {
                d = nullptr;
                return cudaSuccess;
            }
            d = p;
            cudaError_t q = cnt ? cudaMemcpyAsync(p, h, cnt * sizeof(double), cudaMemcpyHostToDevice, s->stream)
                                : cudaSuccess;
            p += cnt;
            return q;
        };
        cudaError_t q = put(x, s->n, dx);
        if (q == cudaSuccess) q = put(lam, s->m, dl);
        if (q == cudaSuccess) q = put(z, s->n, dz);
        if (q == cudaSuccess) q = put(del, s->n, dd);
        if (q != cudaSuccess) {
            cudaFreeAsync(tmp, s->stream);
            return fail(s, MFS_ERR_CUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(q));
        }
    }
    mfs_status st = (s->precision == MFS_FP64) ? warm_start_t(s, s->s64, dx, dl, dz, dd)
                                                : warm_start_t(s, s->s32, dx, dl, dz, dd);
    if (tmp) {
        cudaFreeAsync(tmp, s->stream);
        cudaStreamSynchronize(s->stream);
    }
    return st;
}

// ------------------------------------------------------------------ literal start (Algorithm 1)
static void literal_free(mfs_solver* s) {
    if (!s->lit_mem.empty()) cudaStreamSynchronize(s->stream);
    for (void* p : s->lit_mem) cudaFree(p);
    s->lit_mem.clear();
    s->lit_y = s->lit_g = s->lit_kval = s->lit_w = s->lit_row = nullptr;
    s->lit_krow = s->lit_kcol = s->lit_perm = s->lit_rp = nullptr;
    s->lit_zarg = nullptr;
    s->lit_pending = 0;
}

template <typename P>
mfs_status lit_alloc(mfs_solver* s, P** p, size_t bytes) {
    void* q = nullptr;
    cudaError_t e = mfs::device_malloc(&q, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) return fail(s, MFS_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    s->lit_mem.push_back(q);
    *p = static_cast<P*>(q);
    return MFS_OK;
}

inline int blocks_for(long long count, int bs = 256) {
    return (int)std::max<long long>(1, std::min<long long>((count + bs - 1) / bs, 148LL * 32));
}

// Host arrays (FP64): x, z, delta (n), y, gamma (o, Algorithm 1's nonzero order), lambda (m).
template <typename T>
mfs_status literal_setup(mfs_solver* s, State<T>& st, const double* x, const double* y, const double* z,
                         const double* g, const double* del, const double* lam) {
    literal_free(s);
    const int64_t n = s->n, m = s->m, o = s->o;
    double* tmp = nullptr;
    TRY(lit_alloc(s, &tmp, (size_t)std::max<int64_t>({n, m, o, 1}) * sizeof(double)));
    auto put = [&](const double* h, int64_t cnt, T* dst) -> mfs_status {
        if (!cnt) return MFS_OK;
        CUDA_TRY(s, cudaMemcpyAsync(tmp, h, cnt * sizeof(double), cudaMemcpyHostToDevice, s->stream));
        convert(dst, tmp, cnt, s->stream);
        CUDA_TRY(s, cudaStreamSynchronize(s->stream));  // tmp is reused by the next call
        return MFS_OK;
    };
    T *ly = nullptr, *lg = nullptr, *kval = nullptr;
    TRY(lit_alloc(s, &ly, o * sizeof(T)));
    TRY(lit_alloc(s, &lg, o * sizeof(T)));
    TRY(lit_alloc(s, &kval, o * sizeof(T)));
    s->lit_y = ly;
    s->lit_g = lg;
    s->lit_kval = kval;
    TRY(put(x, n, st.x));
    TRY(put(z, n, st.z));
    TRY(put(del, n, st.del));
    TRY(put(lam, m, st.lam));
    TRY(put(y, o, ly));
    TRY(put(g, o, lg));
    T *w = nullptr, *row = nullptr;
    TRY(lit_alloc(s, &w, o * sizeof(T)));
    TRY(lit_alloc(s, &row, m * sizeof(T)));
    s->lit_w = w;
    s->lit_row = row;
    TRY(lit_alloc(s, &s->lit_krow, o * sizeof(int)));
    TRY(lit_alloc(s, &s->lit_kcol, o * sizeof(int)));
    TRY(lit_alloc(s, &s->lit_perm, o * sizeof(int)));
    TRY(lit_alloc(s, &s->lit_rp, (m + 1) * sizeof(int)));
    TRY(lit_alloc(s, &s->lit_zarg, n * sizeof(double)));
    if (s->ncc)
        mfs::literal::k_kmap<T><<<blocks_for(s->ncc), 256, 0, s->stream>>>(s->col_ptr, s->cdesc, s->ncc, s->cidx,
                                                                          st.cval, s->lit_krow, s->lit_kcol, kval);
    // rows of the k order: a stable counting sort (index bookkeeping of the set-up, as at create)
    std::vector<int> krow(o), rp(m + 1, 0), perm(o);
    if (o) CUDA_TRY(s, cudaMemcpyAsync(krow.data(), s->lit_krow, o * sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(s, cudaStreamSynchronize(s->stream));
    for (int64_t k = 0; k < o; ++k) rp[krow[k] + 1]++;
    for (int64_t i = 0; i < m; ++i) rp[i + 1] += rp[i];
    std::vector<int> fill(rp.begin(), rp.end() - 1);
    for (int64_t k = 0; k < o; ++k) perm[fill[krow[k]]++] = (int)k;
    if (o) CUDA_TRY(s, cudaMemcpyAsync(s->lit_perm, perm.data(), o * sizeof(int), cudaMemcpyHostToDevice, s->stream));
    CUDA_TRY(s, cudaMemcpyAsync(s->lit_rp, rp.data(), (m + 1) * sizeof(int), cudaMemcpyHostToDevice, s->stream));
    CUDA_TRY(s, cudaGetLastError());
    CUDA_TRY(s, cudaStreamSynchronize(s->stream));
    s->lit_pending = 2;
    s->iter = 0;
    return MFS_OK;
}

// One iteration of Algorithm 1 in its literal form.
template <typename T>
mfs_status literal_iteration(mfs_solver* s, State<T>& st) {
    namespace L = mfs::literal;
    const int n = s->n, m = s->m;
    const long long o = s->o;
    const T mu = T(s->set.mu);
    T* y = static_cast<T*>(s->lit_y);
    T* g = static_cast<T*>(s->lit_g);
    T* kval = static_cast<T*>(s->lit_kval);
    T* w = static_cast<T*>(s->lit_w);
    T* row = static_cast<T*>(s->lit_row);
    cudaStream_t q = s->stream;
    if (n) L::k_x<T><<<blocks_for(n), 256, 0, q>>>(s->col_ptr, y, g, st.z, st.del, st.c, mu, st.x, n);
    if (o) L::k_w<T><<<blocks_for(o), 256, 0, q>>>(s->lit_krow, s->lit_kcol, kval, st.b, st.lam, st.x, g, mu, w, o);
    if (m) L::k_rowdot<T><<<blocks_for(m), 256, 0, q>>>(s->lit_rp, s->lit_perm, kval, w, 1, row, m);
    if (o) L::k_y<T><<<blocks_for(o), 256, 0, q>>>(s->lit_krow, kval, w, row, y, o);
    if (n) {
        L::k_zarg<T><<<blocks_for(n), 256, 0, q>>>(st.x, st.del, mu, s->lit_zarg, n);
        k_proj_orthant<T><<<blocks_for(n), 256, 0, q>>>(st.z, s->lit_zarg, n);
        if (s->nsoc)
            k_proj_soc<T><<<blocks_for(s->nsoc), 256, 0, q>>>(st.z, s->lit_zarg, s->soc_start, s->soc_size, s->nsoc);
    }
    if (m) {
        L::k_rowdot<T><<<blocks_for(m), 256, 0, q>>>(s->lit_rp, s->lit_perm, kval, y, 0, row, m);
        L::k_lam<T><<<blocks_for(m), 256, 0, q>>>(row, st.b, mu, st.lam, m);
    }
    if (o) L::k_gam<T><<<blocks_for(o), 256, 0, q>>>(s->lit_kcol, y, st.x, mu, g, o);
    if (n) L::k_del<T><<<blocks_for(n), 256, 0, q>>>(st.z, st.x, mu, st.del, n);
    CUDA_TRY(s, cudaGetLastError());
    return MFS_OK;
}

// Run the pending literal iterations (at most k of them); after the second, switch to the reduced
// state: v = F_U (b - A x) - lambda/mu. Returns the number of iterations run in *done.
template <typename T>
mfs_status literal_run(mfs_solver* s, State<T>& st, int64_t k, int64_t* done) {
    *done = 0;
    while (s->lit_pending > 0 && *done < k) {
        TRY(literal_iteration(s, st));
        --s->lit_pending;
        ++*done;
        ++s->iter;
    }
    if (s->lit_pending == 0 && !s->lit_mem.empty()) {
        launch_warm_v(s, sweep_args(s, st), s->stream);
        CUDA_TRY(s, cudaGetLastError());
        literal_free(s);
    }
    return MFS_OK;
}

// ------------------------------------------------------------------ primal infeasibility test
constexpr int INF_BLOCKS = 296;

// Reductions for the two tests (s_buf and r_buf must hold c + A^T lambda and A x - b of the current
// iterate): out = {dist(A^T d, K)^2, ||d||^2, dist(e, K)^2, ||e||^2, ||A e||^2} with d and e the
// changes of lambda and x since the previous call; then remembers s, lambda, x and r.
template <typename T>
mfs_status infeas_reduce(mfs_solver* s, State<T>& st, bool have_prev, double* out) {
    const int n = s->n, m = s->m, nsoc = s->nsoc;
    if (!s->inf_s_prev) {
        TRY(dalloc(s, &s->inf_s_prev, (size_t)n));
        TRY(dalloc(s, &s->inf_lam_prev, (size_t)m));
        TRY(dalloc(s, &s->inf_x_prev, (size_t)n));
        TRY(dalloc(s, &s->inf_r_prev, (size_t)m));
        TRY(dalloc(s, &s->inf_part, (size_t)5 * INF_BLOCKS + 2 * std::max(nsoc, 1)));
    }
    for (int q = 0; q < 5; ++q) out[q] = 0.0;
    if (have_prev) {
        mfs::infeas::k_infeas<T><<<INF_BLOCKS, 256, 0, s->stream>>>(s->s_buf, s->inf_s_prev, st.lam, s->inf_lam_prev,
                                                                    st.x, s->inf_x_prev, s->r_buf, s->inf_r_prev,
                                                                    s->in_cone, n, m, s->inf_part);
        if (nsoc)
            mfs::infeas::k_infeas_cones<T><<<(nsoc + 255) / 256, 256, 0, s->stream>>>(
                s->s_buf, s->inf_s_prev, st.x, s->inf_x_prev, s->soc_start, s->soc_size, nsoc,
                s->inf_part + 5 * INF_BLOCKS);
        std::vector<double> h(5 * INF_BLOCKS + 2 * nsoc);
        CUDA_TRY(s, cudaMemcpyAsync(h.data(), s->inf_part, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
        CUDA_TRY(s, cudaStreamSynchronize(s->stream));
        for (int b = 0; b < INF_BLOCKS; ++b)
            for (int q = 0; q < 5; ++q) out[q] += h[5 * b + q];
        for (int q = 0; q < nsoc; ++q) {
            out[0] += h[5 * INF_BLOCKS + 2 * q];
            out[2] += h[5 * INF_BLOCKS + 2 * q + 1];
        }
    }
    if (n) {
        CUDA_TRY(s, cudaMemcpyAsync(s->inf_s_prev, s->s_buf, n * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
        convert(s->inf_x_prev, st.x, n, s->stream);
    }
    if (m) {
        convert(s->inf_lam_prev, st.lam, m, s->stream);
        CUDA_TRY(s, cudaMemcpyAsync(s->inf_r_prev, s->r_buf, m * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
    }
    CUDA_TRY(s, cudaGetLastError());
    return MFS_OK;
}

// ====================================================================================== C ABI
namespace mfs {
namespace {
std::atomic<long long> g_alloc_left{-1};  // < 0: no failure armed
}
cudaError_t device_malloc(void** p, size_t bytes) {
    long long left = g_alloc_left.load();
    while (left >= 0) {
        if (left == 0) {
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
        if (g_alloc_left.compare_exchange_weak(left, left - 1)) break;
    }
    return cudaMalloc(p, bytes);
}
}  // namespace mfs

extern "C" {

mfs_status mfs_debug_fail_alloc_after(int64_t n) {
    mfs::g_alloc_left.store(n < 0 ? -1 : (long long)n);
    return MFS_OK;
}


void mfs_default_settings(mfs_settings* st) {
    if (!st) return;
    st->mu = 1.0;
    st->check_every = 25;
    st->precision = MFS_FP64;
    st->polish_iters = 50;
    st->stop_rule = MFS_STOP_KKT;
    st->osqp_rel = 10.0;
    st->sweep = MFS_SWEEP_AUTO;
    st->adapt_mu = 0;
    st->l2_keep = 0;
}

const char* mfs_last_error(const mfs_solver* s) {
    return s ? s->last_error.c_str() : g_create_error.c_str();
}

void mfs_destroy(mfs_solver* s) {
    if (!s) return;
    cudaSetDevice(s->device);
    if (s->stream) cudaStreamSynchronize(s->stream);
    destroy_graphs(s);
    literal_free(s);
    keep_release(s);
    for (void* p : s->allocs) cudaFree(p);
    if (s->h_status) cudaFreeHost(s->h_status);
    if (s->h_err) cudaFreeHost(s->h_err);
    if (s->cap) cudaStreamDestroy(s->cap);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

}  // extern "C"

namespace {

// mfs_create and mfs_create_device: on_device says that row, col, val, b and c are device arrays.
mfs_status create_impl(int64_t m, int64_t n, int64_t nnz, const int64_t* row, const int64_t* col, const double* val,
                       const double* b, const double* c, int64_t ncones, const mfs_cone* cones,
                       const mfs_settings* settings, void* cuda_stream, mfs_solver** out, bool on_device) {
    g_create_error.clear();
    if (!out) return fail(nullptr, MFS_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (m < 0 || n < 0 || nnz < 0 || ncones < 0) return fail(nullptr, MFS_ERR_INVALID, "negative size");
    if (m >= INT32_MAX || n >= INT32_MAX || nnz >= INT32_MAX)
        return fail(nullptr, MFS_ERR_INVALID, "m, n and nnz must be below 2^31");
    if ((nnz && (!row || !col || !val)) || (m && !b) || (n && !c) || (ncones && !cones))
        return fail(nullptr, MFS_ERR_INVALID, "NULL array");
    mfs_settings set;
    mfs_default_settings(&set);
    if (settings) set = *settings;
    if (!(set.mu > 0.0) || !std::isfinite(set.mu)) return fail(nullptr, MFS_ERR_INVALID, "mu must be > 0");
    if (set.check_every < 1) return fail(nullptr, MFS_ERR_INVALID, "check_every must be >= 1");
    if (set.precision != MFS_FP64 && set.precision != MFS_FP32_MIXED)
        return fail(nullptr, MFS_ERR_INVALID, "unknown precision");
    if (set.polish_iters < 0) return fail(nullptr, MFS_ERR_INVALID, "polish_iters must be >= 0");
    if (set.stop_rule != MFS_STOP_KKT && set.stop_rule != MFS_STOP_SCS_L2 && set.stop_rule != MFS_STOP_OSQP_INF)
        return fail(nullptr, MFS_ERR_INVALID, "unknown stop_rule");
    if (!(set.osqp_rel > 0.0) || !std::isfinite(set.osqp_rel))
        return fail(nullptr, MFS_ERR_INVALID, "osqp_rel must be > 0");
    if (set.sweep != MFS_SWEEP_AUTO && set.sweep != MFS_SWEEP_CHUNKED && set.sweep != MFS_SWEEP_STAGED)
        return fail(nullptr, MFS_ERR_INVALID, "unknown sweep kind");
    if (set.adapt_mu < 0) return fail(nullptr, MFS_ERR_INVALID, "adapt_mu must be >= 0");
    if (set.l2_keep != 0 && set.l2_keep != 1) return fail(nullptr, MFS_ERR_INVALID, "l2_keep must be 0 or 1");
    int64_t total = 0;
    for (int64_t q = 0; q < ncones; ++q) {
        if (cones[q].size < 1) return fail(nullptr, MFS_ERR_INVALID, "cone of size < 1");
        if (cones[q].kind != MFS_CONE_NONNEG && cones[q].kind != MFS_CONE_SOC)
            return fail(nullptr, MFS_ERR_INVALID, "unknown cone kind");
        total += cones[q].size;
    }
    if (total != n) return fail(nullptr, MFS_ERR_INVALID, "cone sizes do not sum to n");
    bool in_order = false;
    // large inputs are checked and, when already in column order, set up on the GPU (the staged
    // layout too); so is every input that is already on the device
    const bool dev_path = on_device || nnz >= (int64_t(1) << 16);
    if (!dev_path) {
        // first bad entry: index out of range, or a non-finite value; and whether the entries are
        // already in (column, row) order (equal neighbours are duplicates, summed later)
        const int nt = mfs::host::threads_for(nnz);
        std::vector<int64_t> bad_idx(nt, nnz), bad_val(nt, nnz);
        std::vector<char> unsorted(nt, 0);
        mfs::host::parallel_ranges(nnz, nt, [&](int64_t lo, int64_t hi, int t) {
            for (int64_t q = lo; q < hi; ++q) {
                if (bad_idx[t] == nnz && (row[q] < 0 || row[q] >= m || col[q] < 0 || col[q] >= n)) bad_idx[t] = q;
                if (bad_val[t] == nnz && !std::isfinite(val[q])) bad_val[t] = q;
                if (q + 1 < nnz && (col[q] > col[q + 1] || (col[q] == col[q + 1] && row[q] > row[q + 1])))
                    unsorted[t] = 1;
            }
        });
        in_order = std::find(unsorted.begin(), unsorted.end(), 1) == unsorted.end();
        const int64_t bi = *std::min_element(bad_idx.begin(), bad_idx.end());
        const int64_t bv = *std::min_element(bad_val.begin(), bad_val.end());
        if (bi < nnz && bi <= bv)
            return fail(nullptr, MFS_ERR_INVALID, "COO index out of range at entry " + std::to_string(bi));
        if (bv < nnz) return fail(nullptr, MFS_ERR_INVALID, "non-finite value in A");
    }
    if (!on_device && (!finite_all(b, m) || !finite_all(c, n)))
        return fail(nullptr, MFS_ERR_INVALID, "non-finite value in b or c");

    mfs_solver* s = new (std::nothrow) mfs_solver();
    if (!s) return fail(nullptr, MFS_ERR_OOM, "host allocation failed");
    auto bail = [&](mfs_status st) {
        g_create_error = s->last_error;
        mfs_destroy(s);
        return st;
    };
    s->set = set;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess) {
        s->last_error = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return bail(MFS_ERR_CUDA);
    }
    if (cuda_stream) {
        s->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            s->last_error = std::string("cudaStreamCreate: ") + cudaGetErrorString(e);
            return bail(MFS_ERR_CUDA);
        }
        s->own_stream = true;
    }
    e = cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        s->last_error = std::string("cudaStreamCreate: ") + cudaGetErrorString(e);
        return bail(MFS_ERR_CUDA);
    }
    if (on_device) {
        // b and c: checked on the device
        int* flag = nullptr;
        mfs_status q = dalloc(s, &flag, 1);
        if (q != MFS_OK) return bail(q);
        int h = 0;
        e = cudaMemsetAsync(flag, 0, sizeof(int), s->stream);
        const int grid = 8 * 148;
        if (e == cudaSuccess && m > 0) mfs::setup::k_nonfinite<<<grid, 256, 0, s->stream>>>(b, m, flag);
        if (e == cudaSuccess && n > 0) mfs::setup::k_nonfinite<<<grid, 256, 0, s->stream>>>(c, n, flag);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) {
            s->last_error = std::string("checking b and c: ") + cudaGetErrorString(e);
            return bail(MFS_ERR_CUDA);
        }
        if (h) {
            s->last_error = "non-finite value in b or c";
            return bail(MFS_ERR_INVALID);
        }
    }
    HostProblem P;
    mfs_status st = MFS_OK;
    // device COO that is not in column order is ordered on the host: these hold its copy
    std::vector<int64_t> h_row, h_col;
    std::vector<double> h_val;
    if (dev_path) {
        st = device_orders(s, m, n, nnz, row, col, val, P, on_device);
        if (st != MFS_OK) return bail(st);
        if (on_device && !P.dev.on) {
            h_row.resize(nnz);
            h_col.resize(nnz);
            h_val.resize(nnz);
            e = cudaSuccess;
            if (nnz > 0) {
                e = cudaMemcpyAsync(h_row.data(), row, nnz * sizeof(int64_t), cudaMemcpyDeviceToHost, s->stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(h_col.data(), col, nnz * sizeof(int64_t), cudaMemcpyDeviceToHost, s->stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(h_val.data(), val, nnz * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
            }
            if (e != cudaSuccess) {
                s->last_error = std::string("copying the COO to the host: ") + cudaGetErrorString(e);
                return bail(MFS_ERR_CUDA);
            }
            row = h_row.data();
            col = h_col.data();
            val = h_val.data();
        }
    }
    st = setup_host(s, m, n, nnz, row, col, val, in_order, ncones, cones, P);
    if (st != MFS_OK) return bail(st);
    s->m = P.m;
    s->n = P.n;
    s->o = P.o;
    s->ncones = (int)ncones;
    s->nsoc = (int)P.soc_start.size();
    s->nbig = (int)P.big_list.size();
    s->has_soc = s->nsoc > 0;
    s->ncc = P.cc.count();
    s->nrc = P.rc.count();
    s->cpad = P.cc.padded;
    s->rpad = P.rc.padded;
    s->nlc = (int)P.cc.longs.size();
    s->nlr = (int)P.rc.longs.size();
    s->precision = set.precision;

#define CHK(x)                      \
    do {                            \
        mfs_status q_ = (x);        \
        if (q_ != MFS_OK) return bail(q_); \
    } while (0)
    CHK(upload(s, &s->col_ptr, P.col_ptr.data(), P.col_ptr.size()));
    CHK(upload(s, &s->row_ptr, P.row_ptr.data(), P.row_ptr.size()));
    CHK(upload(s, reinterpret_cast<int**>(&s->cdesc), P.cc.desc.data(), P.cc.desc.size()));
    CHK(upload(s, reinterpret_cast<int**>(&s->rdesc), P.rc.desc.data(), P.rc.desc.size()));
    CHK(upload(s, &s->cheads, P.cc.heads.data(), P.cc.heads.size()));
    CHK(upload(s, &s->rheads, P.rc.heads.data(), P.rc.heads.size()));
    CHK(upload(s, &s->clong, P.cc.longs.data(), P.cc.longs.size()));
    CHK(upload(s, &s->rlong, P.rc.longs.data(), P.rc.longs.size()));
    CHK(upload(s, &s->cq_lo, P.cq_lo.data(), P.cq_lo.size()));
    CHK(upload(s, &s->cq_hi, P.cq_hi.data(), P.cq_hi.size()));
    CHK(upload(s, &s->soc_start, P.soc_start.data(), P.soc_start.size()));
    CHK(upload(s, &s->soc_size, P.soc_size.data(), P.soc_size.size()));
    {
        std::vector<unsigned char> inc(n, 0);
        for (size_t q = 0; q < P.soc_start.size(); ++q)
            for (int t = 0; t < P.soc_size[q]; ++t) inc[P.soc_start[q] + t] = P.soc_big[q] ? 2 : 1;
        CHK(upload(s, &s->in_cone, inc.data(), inc.size()));
    }
    CHK(upload(s, &s->soc_big, P.soc_big.data(), P.soc_big.size()));
    CHK(upload(s, &s->big_list, P.big_list.data(), P.big_list.size()));
    {
        // padded index arrays (shared by both precisions)
        if (P.dev.on) {
            CHK(pad_on_device<float>(s, P, true, &s->cidx, nullptr));
            CHK(pad_on_device<float>(s, P, false, &s->ridx, nullptr));
        } else {
            mfs::host::uvec<int> pidx;
            pad_chunks<double>(P.cc, P.col_ptr, P.csc_row, P.csc_val, &pidx, (mfs::host::uvec<double>*)nullptr);
            CHK(upload(s, &s->cidx, pidx.data(), pidx.size()));
            pad_chunks<double>(P.rc, P.row_ptr, P.csr_col, P.csr_val, &pidx, (mfs::host::uvec<double>*)nullptr);
            CHK(upload(s, &s->ridx, pidx.data(), pidx.size()));
        }
    }
    {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device) == cudaSuccess && sms > 0)
            s->num_sms = sms;
    }
    if (set.precision == MFS_FP32_MIXED) {
        CHK(alloc_state<float>(s, s->s32, P, b, c, on_device));
        CHK(residual_grids<float>(s));
        s->have32 = true;
        // what the automatic choice stages (the same whether or not it is the creation's choice)
        const bool big = P.dev.on && P.o >= (1 << 20);
        const bool auto_col = big && (int64_t)P.o >= 8 * (int64_t)P.m;
        const bool auto_row = big && (int64_t)P.o >= 4 * (int64_t)P.n;
        if ((set.sweep == MFS_SWEEP_STAGED || (set.sweep == MFS_SWEEP_AUTO && (auto_col || auto_row))) && P.o > 0)
            CHK(setup_staged(s, P));
        s->stg_auto_col = s->stg_ok && auto_col;
        s->stg_auto_row = s->stg_ok && auto_row;
        s->sweep_kind = s->stg_ok ? set.sweep : MFS_SWEEP_AUTO;
    }
    if (set.precision == MFS_FP64 || set.polish_iters > 0) {
        CHK(alloc_state<double>(s, s->s64, P, b, c, on_device));
        CHK(residual_grids<double>(s));
        s->have64 = true;
    }
    CHK(dalloc(s, &s->part_row, (size_t)s->g_rowres * NFR));
    CHK(dalloc(s, &s->part_col, (size_t)s->g_colres * NFC));
    CHK(dalloc(s, &s->part_big, (size_t)std::max(s->nbig, 1) * NFB));
    CHK(dalloc(s, &s->s_buf, (size_t)std::max(s->n, 1)));
    CHK(dalloc(s, &s->r_buf, (size_t)std::max(s->m, 1)));
    CHK(dalloc(s, &s->status, NSTATUS));
    e = cudaMallocHost(&s->h_status, NSTATUS * sizeof(double));
    if (e != cudaSuccess) {
        s->last_error = std::string("pinned allocation: ") + cudaGetErrorString(e);
        return bail(MFS_ERR_CUDA);
    }
    e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        s->last_error = std::string("set-up: ") + cudaGetErrorString(e);
        return bail(MFS_ERR_CUDA);
    }
#undef CHK
    *out = s;
    return MFS_OK;
}

}  // namespace

extern "C" {

mfs_status mfs_create(int64_t m, int64_t n, int64_t nnz, const int64_t* row, const int64_t* col, const double* val,
                      const double* b, const double* c, int64_t ncones, const mfs_cone* cones,
                      const mfs_settings* settings, void* cuda_stream, mfs_solver** out) {
    MFS_TRACE("mfs_create");
    return create_impl(m, n, nnz, row, col, val, b, c, ncones, cones, settings, cuda_stream, out, false);
}

mfs_status mfs_create_device(int64_t m, int64_t n, int64_t nnz, const int64_t* row, const int64_t* col,
                             const double* val, const double* b, const double* c, int64_t ncones,
                             const mfs_cone* cones, const mfs_settings* settings, void* cuda_stream,
                             mfs_solver** out) {
    MFS_TRACE("mfs_create_device");
    return create_impl(m, n, nnz, row, col, val, b, c, ncones, cones, settings, cuda_stream, out, true);
}

mfs_status mfs_get_info(const mfs_solver* s, mfs_info_t* out) {
    if (!s || !out) return MFS_ERR_INVALID;
    out->m = s->m;
    out->n = s->n;
    out->o = s->o;
    out->ncones = s->ncones;
    out->nsoc = s->nsoc;
    out->nbig = s->nbig;
    out->col_chunks = s->ncc;
    out->row_chunks = s->nrc;
    out->bytes_per_iter = bytes_per_iter(s, s->precision);
    out->precision = s->precision;
    out->launches_per_iter = launches_per_iteration(s);
    const bool f32 = s->precision == MFS_FP32_MIXED;
    out->sweep_col = (f32 && staged_col(s)) ? MFS_SWEEP_STAGED : MFS_SWEEP_CHUNKED;
    out->sweep_row = (f32 && staged_row(s)) ? MFS_SWEEP_STAGED : MFS_SWEEP_CHUNKED;
    out->col_parts = s->stg_ok ? s->stg_col.halves : 0;
    out->row_parts = s->stg_ok ? s->stg_row.halves : 0;
    return MFS_OK;
}

mfs_status mfs_debug_staged_wait_test(mfs_solver* s) {
    if (!s) return MFS_ERR_INVALID;
    if (!s->stg_ok) return fail(s, MFS_ERR_INVALID, "no staged sweeps on this solver");
    CUDA_TRY(s, cudaSetDevice(s->device));
    StagedArgsT g = s->stg_col;
    g.spin = 64;
    g.no_loads = 1;
    const SweepArgs<float> a = sweep_args(s, s->s32);
    const size_t smem = mfs::staged::smem_bytes(mfs::staged::RB_COL, mfs::staged::S_COL, g.maxg_pad, g.R);
    if (s->has_soc)
        MFS_STAGED_COL_SOC<<<std::min(g.G, s->num_sms), mfs::staged::NTHREADS, smem, s->stream>>>(g, a);
    else
        MFS_STAGED_COL<<<std::min(g.G, s->num_sms), mfs::staged::NTHREADS, smem, s->stream>>>(g, a);
    CUDA_TRY(s, cudaGetLastError());
    CUDA_TRY(s, cudaMemcpyAsync(s->h_err, s->stg_err, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(s, cudaMemsetAsync(s->stg_err, 0, sizeof(int), s->stream));
    CUDA_TRY(s, cudaStreamSynchronize(s->stream));
    const int flagged = *s->h_err;
    *s->h_err = 0;
    return flagged ? fail(s, MFS_ERR_TIMEOUT, "staged sweep: wait for a block gave up (diagnostic)") : MFS_OK;
}

int32_t mfs_debug_bounds(int64_t* site, int64_t* index, int32_t reset) {
#ifdef MFS_DEBUG_BOUNDS
    unsigned long long v = 0;
    cudaDeviceSynchronize();
    cudaMemcpyFromSymbol(&v, mfs::g_bounds_fail, sizeof v);
    const unsigned long long vs = mfs::static_bounds_record(reset != 0);
    if (v == 0) v = vs;
    if (site) *site = (int64_t)(v >> 40);
    if (index) *index = (int64_t)(v & 0xFFFFFFFFFFull);
    if (reset) {
        const unsigned long long zero = 0;
        cudaMemcpyToSymbol(mfs::g_bounds_fail, &zero, sizeof zero);
    }
    return 1;
#else
    (void)reset;
    if (site) *site = 0;
    if (index) *index = 0;
    return 0;
#endif
}

mfs_status mfs_set_sweep(mfs_solver* s, int32_t kind) {
    if (!s) return MFS_ERR_INVALID;
    if (kind != MFS_SWEEP_AUTO && kind != MFS_SWEEP_CHUNKED && kind != MFS_SWEEP_STAGED)
        return fail(s, MFS_ERR_INVALID, "unknown sweep kind");
    if (kind == MFS_SWEEP_STAGED && !s->stg_ok)
        return fail(s, MFS_ERR_INVALID,
                    "no staged layout: create the solver with settings.sweep = MFS_SWEEP_STAGED (FP32_MIXED)");
    CUDA_TRY(s, cudaSetDevice(s->device));
    CUDA_TRY(s, cudaStreamSynchronize(s->stream));
    destroy_graphs(s);
    s->sweep_kind = kind;
    return MFS_OK;
}

mfs_status mfs_set_mu(mfs_solver* s, double mu) {
    if (!s) return MFS_ERR_INVALID;
    if (!(mu > 0.0) || !std::isfinite(mu)) return fail(s, MFS_ERR_INVALID, "mu must be > 0");
    CUDA_TRY(s, cudaSetDevice(s->device));
    const double old = s->set.mu;
    s->set.mu = mu;
    destroy_graphs(s);  // mu is baked into the captured launches
    if (old == mu) return MFS_OK;
    // v = rho - lambda/mu depends on mu. rho = F_U (b - A x) is recomputed from the current x by
    // the same row-order kernel that produced it, so only the lambda/mu term changes.
    if (s->precision == MFS_FP64)
        launch_warm_v(s, sweep_args(s, s->s64), s->stream);
    else
        launch_warm_v(s, sweep_args(s, s->s32), s->stream);
    CUDA_TRY(s, cudaGetLastError());
    CUDA_TRY(s, cudaStreamSynchronize(s->stream));
    return MFS_OK;
}

mfs_status mfs_warm_start(mfs_solver* s, const double* x, const double* lambda, const double* z,
                          const double* delta) {
    return warm_start_impl(s, x, lambda, z, delta, true);
}

mfs_status mfs_warm_start_literal(mfs_solver* s, const double* x, const double* y, const double* z,
                                  const double* gamma, const double* delta, const double* lambda) {
    if (!s) return MFS_ERR_INVALID;
    if ((s->n && (!x || !z || !delta)) || (s->o && (!y || !gamma)) || (s->m && !lambda))
        return fail(s, MFS_ERR_INVALID, "x, y, z, gamma, delta and lambda are all required");
    CUDA_TRY(s, cudaSetDevice(s->device));
    mfs_status st = s->precision == MFS_FP64 ? literal_setup(s, s->s64, x, y, z, gamma, delta, lambda)
                                              : literal_setup(s, s->s32, x, y, z, gamma, delta, lambda);
    if (st != MFS_OK) literal_free(s);
    return st;
}

mfs_status mfs_warm_start_device(mfs_solver* s, const double* x, const double* lambda, const double* z,
                                 const double* delta) {
    return warm_start_impl(s, x, lambda, z, delta, false);
}

mfs_status mfs_iterate(mfs_solver* s, int64_t k) {
    MFS_TRACE("mfs_iterate");
    if (!s) return MFS_ERR_INVALID;
    if (k < 0) return fail(s, MFS_ERR_INVALID, "k must be >= 0");
    CUDA_TRY(s, cudaSetDevice(s->device));
    if (s->lit_pending > 0) {
        int64_t done = 0;
        TRY(s->precision == MFS_FP64 ? literal_run(s, s->s64, k, &done) : literal_run(s, s->s32, k, &done));
        k -= done;
    }
    TRY(s->precision == MFS_FP64 ? run_iters(s, s->s64, k) : run_iters(s, s->s32, k));
    CUDA_TRY(s, cudaStreamSynchronize(s->stream));
    return MFS_OK;
}

mfs_status mfs_residuals(mfs_solver* s, mfs_residuals_t* out) {
    MFS_TRACE("mfs_residuals");
    if (!s || !out) return MFS_ERR_INVALID;
    CUDA_TRY(s, cudaSetDevice(s->device));
    return s->precision == MFS_FP64 ? residuals_t(s, s->s64, out, false) : residuals_t(s, s->s32, out, false);
}

mfs_status mfs_set_precision(mfs_solver* s, int32_t precision) {
    if (!s) return MFS_ERR_INVALID;
    if (precision != MFS_FP64 && precision != MFS_FP32_MIXED) return fail(s, MFS_ERR_INVALID, "unknown precision");
    if (precision == s->precision) return MFS_OK;
    if (s->lit_pending > 0)
        return fail(s, MFS_ERR_INVALID, "a literal start is pending: iterate twice before changing the precision");
    if ((precision == MFS_FP64 && !s->have64) || (precision == MFS_FP32_MIXED && !s->have32))
        return fail(s, MFS_ERR_INVALID, "that precision was not prepared at mfs_create");
    CUDA_TRY(s, cudaSetDevice(s->device));
    if (precision == MFS_FP64)
        copy_state(s, s->s64, s->s32);
    else
        copy_state(s, s->s32, s->s64);
    s->precision = precision;
    CUDA_TRY(s, cudaGetLastError());
    CUDA_TRY(s, cudaStreamSynchronize(s->stream));
    return MFS_OK;
}

mfs_status mfs_solve(mfs_solver* s, double tol, int64_t max_iter, int64_t* iters_out) {
    if (!s) return MFS_ERR_INVALID;
    MFS_TRACE("mfs_solve");
    constexpr int64_t HIST_CAP = 4096;
    s->hist.assign(HIST_CAP, mfs_check_t{});
    s->hist_count = 0;
    if (!(tol > 0.0) || max_iter < 0) return fail(s, MFS_ERR_INVALID, "tol must be > 0 and max_iter >= 0");
    CUDA_TRY(s, cudaSetDevice(s->device));
    const int64_t K = s->set.check_every;
    int64_t it = 0;
    double best = std::numeric_limits<double>::infinity();
    int since_best = 0;
    mfs_residuals_t r;
    mfs_status result = MFS_MAX_ITER;
    // infeasibility tests: previous b^T lambda, c^T x and precision, consecutive passes, and the
    // primal and dual residuals of the last checks
    bool have_prev = false;
    int prev_prec = -1, pass_p = 0, pass_d = 0;
    double prev_blam = 0.0, prev_cx = 0.0;
    std::vector<double> rp_hist, rd_hist;
    // residual balancing of mu (settings.adapt_mu > 0): the factor, the imbalance that triggers it
    // and the range around the starting mu
    constexpr double MU_STEP = 2.0, MU_TAU = 5.0, MU_RANGE = 256.0;
    const double mu0 = s->set.mu;
    int64_t nchk = 0;  // checks made by this call before the current one
    int64_t next_adapt = s->set.adapt_mu;  // the next check that may change mu
    while (true) {
        TRY(s->precision == MFS_FP64 ? residuals_t(s, s->s64, &r, true) : residuals_t(s, s->s32, &r, true));
        const double meas = stop_measure(r, s->set.stop_rule);
        {
            mfs_check_t& h = s->hist[(size_t)(s->hist_count % HIST_CAP)];
            h.iter = it;
            h.kkt = r.kkt;
            h.r_prim = r.r_prim;
            h.r_dual = r.r_dual;
            h.r_cone = r.r_cone;
            h.r_gap = r.r_gap;
            h.measure = meas;
            h.precision = s->precision;
            h.reserved = 0;
            h.mu = s->set.mu;
            ++s->hist_count;
        }
        if (!std::isfinite(r.kkt) || !std::isfinite(meas)) {
            result = fail(s, MFS_ERR_NUMERIC, "NaN or Inf in the residuals");
            break;
        }
        {
            double red[5];
            const bool same = have_prev && prev_prec == s->precision;
            TRY(s->precision == MFS_FP64 ? infeas_reduce(s, s->s64, same, red) : infeas_reduce(s, s->s32, same, red));
            const double blam = -r.dobj, cx = r.pobj;  // b^T lambda, c^T x
            rp_hist.push_back(r.r_prim);
            rd_hist.push_back(r.r_dual);
            if (same && meas > tol) {
                const size_t h = rp_hist.size();
                // primal infeasible: d = change of lambda, A^T d in K, b^T d < 0
                const double bd = blam - prev_blam;
                const bool p_stall = h >= 4 && rp_hist[h - 1] >= 0.99 * rp_hist[h - 4];
                const bool p_pass = bd < -1e-3 * r.nrm_b * std::sqrt(red[1]) && std::sqrt(red[0]) <= 0.1 * -bd && p_stall;
                pass_p = p_pass ? pass_p + 1 : 0;
                // unbounded: e = change of x, A e = 0, e in K, c^T e < 0
                const double ce = cx - prev_cx;
                const bool d_stall = h >= 4 && rd_hist[h - 1] >= 0.99 * rd_hist[h - 4];
                const bool d_pass = ce < -1e-3 * r.nrm_c * std::sqrt(red[3]) && std::sqrt(red[4]) <= 0.1 * -ce &&
                                    std::sqrt(red[2]) <= 0.1 * -ce && d_stall;
                pass_d = d_pass ? pass_d + 1 : 0;
                if (pass_p >= 3) {
                    result = fail(s, MFS_INFEASIBLE, "primal infeasibility certificate (Farkas) found");
                    break;
                }
                if (pass_d >= 3) {
                    result = fail(s, MFS_UNBOUNDED, "a ray of the primal with falling cost found (the dual is infeasible)");
                    break;
                }
            }
            have_prev = true;
            prev_prec = s->precision;
            prev_blam = blam;
            prev_cx = cx;
        }
        const bool fp32 = s->precision == MFS_FP32_MIXED;
        if (meas <= tol) {
            if (fp32 && s->have64 && s->set.polish_iters > 0 && it < max_iter) {
                TRY(mfs_set_precision(s, MFS_FP64));
                const int64_t p = std::min<int64_t>(s->set.polish_iters, max_iter - it);
                TRY(mfs_iterate(s, p));
                it += p;
                ++nchk;
                continue;  // re-check in FP64
            }
            result = MFS_OK;
            break;
        }
        if (it >= max_iter) break;
        if (fp32 && s->have64) {
            if (meas < 0.99 * best) {
                best = meas;
                since_best = 0;
            } else if (++since_best >= 40) {
                TRY(mfs_set_precision(s, MFS_FP64));
            }
        }
        if (s->set.adapt_mu > 0 && nchk == next_adapt) {
            next_adapt *= 2;  // exponentially spaced changes: finitely many over any run
            // residual balancing (a variant outside the paper, which keeps mu fixed)
            const double rp = std::max(r.r_prim, r.r_cone), rd = r.r_dual;
            double mu = s->set.mu;
            if (rp > MU_TAU * rd)
                mu *= MU_STEP;
            else if (rd > MU_TAU * rp)
                mu /= MU_STEP;
            mu = std::min(std::max(mu, mu0 / MU_RANGE), mu0 * MU_RANGE);
            if (mu != s->set.mu) {
                TRY(mfs_set_mu(s, mu));
                s->hist[(size_t)((s->hist_count - 1) % HIST_CAP)].mu = mu;
            }
        }
        ++nchk;
        const int64_t kk = std::min<int64_t>(K, max_iter - it);
        TRY(mfs_iterate(s, kk));
        it += kk;
    }
    if (iters_out) *iters_out = it;
    return result;
}

mfs_status mfs_solve_history(const mfs_solver* s, mfs_check_t* out, int64_t capacity, int64_t* count) {
    if (!s || capacity < 0 || (capacity > 0 && !out)) return MFS_ERR_INVALID;
    const int64_t cap = (int64_t)s->hist.size();
    const int64_t kept = std::min(s->hist_count, cap);
    const int64_t give = std::min(kept, capacity);
    const int64_t first = s->hist_count - give;  // the most recent `give` checks, oldest first
    for (int64_t q = 0; q < give; ++q) out[q] = s->hist[(size_t)((first + q) % cap)];
    if (count) *count = s->hist_count;
    return MFS_OK;
}

mfs_status mfs_get_solution(mfs_solver* s, double* x, double* lambda, double* z, double* delta) {
    if (!s) return MFS_ERR_INVALID;
    CUDA_TRY(s, cudaSetDevice(s->device));
    return s->precision == MFS_FP64 ? get_solution_t(s, s->s64, x, lambda, z, delta, true)
                                    : get_solution_t(s, s->s32, x, lambda, z, delta, true);
}

mfs_status mfs_get_solution_device(mfs_solver* s, double* x, double* lambda, double* z, double* delta) {
    if (!s) return MFS_ERR_INVALID;
    CUDA_TRY(s, cudaSetDevice(s->device));
    return s->precision == MFS_FP64 ? get_solution_t(s, s->s64, x, lambda, z, delta, false)
                                    : get_solution_t(s, s->s32, x, lambda, z, delta, false);
}

mfs_status mfs_get_reduced_v(mfs_solver* s, double* v) {
    if (!s || (!v && s->m > 0)) return MFS_ERR_INVALID;
    if (s->lit_pending > 0) return fail(s, MFS_ERR_INVALID, "a literal start is pending: v is not formed yet");
    CUDA_TRY(s, cudaSetDevice(s->device));
    if (s->m == 0) return MFS_OK;
    double* tmp = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&tmp, (size_t)s->m * sizeof(double), s->stream);
    if (e != cudaSuccess) return fail(s, MFS_ERR_OOM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
    if (s->precision == MFS_FP64)
        convert(tmp, s->s64.v, s->m, s->stream);
    else
        convert(tmp, s->s32.v, s->m, s->stream);
    e = cudaMemcpyAsync(v, tmp, (size_t)s->m * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    cudaFreeAsync(tmp, s->stream);
    if (e != cudaSuccess) return fail(s, MFS_ERR_CUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
    CUDA_TRY(s, cudaStreamSynchronize(s->stream));
    return MFS_OK;
}

mfs_status mfs_time_kernel_split(mfs_solver* s, int64_t k, double* out_ms) {
    if (!s || !out_ms || k < 0) return MFS_ERR_INVALID;
    CUDA_TRY(s, cudaSetDevice(s->device));
    return s->precision == MFS_FP64 ? time_kernels_t(s, s->s64, k, out_ms, true)
                                    : time_kernels_t(s, s->s32, k, out_ms, true);
}

mfs_status mfs_time_kernels(mfs_solver* s, int64_t k, double* out_ms) {
    if (!s || !out_ms || k < 0) return MFS_ERR_INVALID;
    CUDA_TRY(s, cudaSetDevice(s->device));
    double t[6];
    const mfs_status r = s->precision == MFS_FP64 ? time_kernels_t(s, s->s64, k, t, false)
                                                  : time_kernels_t(s, s->s32, k, t, false);
    if (r != MFS_OK) return r;
    out_ms[0] = t[0] + t[1];
    out_ms[1] = t[3] + t[4];
    out_ms[2] = t[2];
    out_ms[3] = t[5];
    return MFS_OK;
}

}  // extern "C"
