// mfs_static.cu -- mfs_row_residuals_static: the row-order FP64 residual reduction for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they want a residual: code that runs
// while another framework owns every byte of device memory through its own pool (and forbids
// side allocations), plugin-style hosts whose execute callbacks must not allocate, or
// real-time loops that allow allocation only at start-up. For them this entry point evaluates
// the row-side residual quantities of a point (x, lambda) for a CSR matrix they already hold on
// the device, with its per-CTA scratch in a fixed static device array instead of memory from
// mfs_create or cudaMalloc.
//
// Scratch: one row of NPART doubles per CTA of ROWS_PER_CTA rows, at most MAX_CTAS CTAs, so
// m <= MAX_CTAS * ROWS_PER_CTA rows (4,194,304); 1 MiB that every GPU which loads this library
// holds until the process exits. All calls share it: calls whose work overlaps on the GPU (for
// example on two streams) race on it and must be serialized by the caller. Nothing in it has to
// start at zero: each call's first kernel writes every slot that its second kernel reads.
// The array's device address is taken in the caller's current context at every call that is not
// being captured into a CUDA graph; a call made during a capture reuses the address of the last
// call in the same context, so one call per context must come before capturing one.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/mfs.h"
#include "mfs_alloc.h"
#include "mfs_device.cuh"
#include "mfs_host.h"

namespace {

constexpr int RS_NT = 256;                      // threads per CTA
constexpr int RS_ROWS_PER_CTA = 256;            // rows per CTA (one warp takes every 8th row)
constexpr int RS_MAX_CTAS = 16384;              // scratch rows
constexpr int RS_NPART = 8;                     // doubles per scratch row (6 used)
constexpr int RS_MAX_DEVICES = 64;

enum : int { P_RES2 = 0, P_RESMAX, P_AXMAX, P_B2, P_BMAX, P_BLAM };

static __device__ __align__(256) double g_row_resid_scratch[RS_MAX_CTAS * RS_NPART];

// The array's device address belongs to a CUDA context: it is looked up again on every call that
// is not being captured into a graph, and kept per device together with the context it was taken
// in, for calls made while their stream is captured (which must not call into module loading).
std::mutex g_setup_mutex;
double* g_scratch_addr[RS_MAX_DEVICES] = {};
CUcontext g_scratch_ctx[RS_MAX_DEVICES] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext*);

CUcontext current_context() {
    static CtxGetCurrentFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<CtxGetCurrentFn>(p);
    }();
    CUcontext c = nullptr;
    if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
    return c;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    return v;
}

// Per-CTA partials: sum (Ax-b)^2, max |Ax-b|, max |Ax|, sum b^2, max |b|, sum b*lambda over the
// CTA's rows, FP64, one warp per row, fixed order (deterministic).
__global__ void __launch_bounds__(RS_NT) k_row_resid_static(int m, int n, const int* __restrict__ row_ptr,
                                                            const int* __restrict__ col_idx,
                                                            const double* __restrict__ val,
                                                            const double* __restrict__ b,
                                                            const double* __restrict__ x,
                                                            const double* __restrict__ lam, double* scratch) {
    __shared__ double sh[RS_NT / 32][6];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r0 = blockIdx.x * RS_ROWS_PER_CTA;
#ifdef MFS_DEBUG_BOUNDS
    const int nnz = row_ptr[m];
#endif
    double f[6] = {0, 0, 0, 0, 0, 0};
    for (int rl = warp; rl < RS_ROWS_PER_CTA; rl += RS_NT / 32) {
        const int i = r0 + rl;
        if (i >= m) break;
        double ax = 0.0;
        for (int k = row_ptr[i] + lane; k < row_ptr[i + 1]; k += 32) {
            if (!MFS_INB(k, nnz, ::mfs::BS_STATIC_ENT)) continue;  // checked build: record and skip
            const int j = col_idx[k];
            if (MFS_INB(j, n, ::mfs::BS_STATIC_X)) ax += val[k] * x[j];
        }
        ax = warp_sum(ax);
        const double bi = b[i], res = ax - bi;
        f[P_RES2] += res * res;
        f[P_RESMAX] = fmax(f[P_RESMAX], fabs(res));
        f[P_AXMAX] = fmax(f[P_AXMAX], fabs(ax));
        f[P_B2] += bi * bi;
        f[P_BMAX] = fmax(f[P_BMAX], fabs(bi));
        f[P_BLAM] += bi * lam[i];
    }
    if (lane == 0)
        for (int t = 0; t < 6; ++t) sh[warp][t] = f[t];
    __syncthreads();
    if (threadIdx.x == 0) {
        double g[6] = {0, 0, 0, 0, 0, 0};
        for (int w = 0; w < RS_NT / 32; ++w) {
            g[P_RES2] += sh[w][P_RES2];
            g[P_RESMAX] = fmax(g[P_RESMAX], sh[w][P_RESMAX]);
            g[P_AXMAX] = fmax(g[P_AXMAX], sh[w][P_AXMAX]);
            g[P_B2] += sh[w][P_B2];
            g[P_BMAX] = fmax(g[P_BMAX], sh[w][P_BMAX]);
            g[P_BLAM] += sh[w][P_BLAM];
        }
        double* out = scratch + (size_t)blockIdx.x * RS_NPART;
        for (int t = 0; t < 6; ++t) out[t] = g[t];
    }
}

// One CTA folds the partials in a fixed order and writes
// out[0..7] = {r_prim, ||Ax-b||_2, ||Ax-b||_inf, ||Ax||_inf, ||b||_2, ||b||_inf, b^T lambda, -b^T lambda}.
__global__ void __launch_bounds__(RS_NT) k_row_resid_static_finalize(int nparts, const double* scratch,
                                                                     double* out) {
    __shared__ double sh[RS_NT][6];
    double f[6] = {0, 0, 0, 0, 0, 0};
    for (int p = threadIdx.x; p < nparts; p += RS_NT) {
        const double* q = scratch + (size_t)p * RS_NPART;
        f[P_RES2] += q[P_RES2];
        f[P_RESMAX] = fmax(f[P_RESMAX], q[P_RESMAX]);
        f[P_AXMAX] = fmax(f[P_AXMAX], q[P_AXMAX]);
        f[P_B2] += q[P_B2];
        f[P_BMAX] = fmax(f[P_BMAX], q[P_BMAX]);
        f[P_BLAM] += q[P_BLAM];
    }
    for (int t = 0; t < 6; ++t) sh[threadIdx.x][t] = f[t];
    __syncthreads();
    for (int s = RS_NT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            double* a = sh[threadIdx.x];
            const double* c = sh[threadIdx.x + s];
            a[P_RES2] += c[P_RES2];
            a[P_RESMAX] = fmax(a[P_RESMAX], c[P_RESMAX]);
            a[P_AXMAX] = fmax(a[P_AXMAX], c[P_AXMAX]);
            a[P_B2] += c[P_B2];
            a[P_BMAX] = fmax(a[P_BMAX], c[P_BMAX]);
            a[P_BLAM] += c[P_BLAM];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double* a = sh[0];
        const double nres = sqrt(a[P_RES2]), nb = sqrt(a[P_B2]);
        out[0] = nres / (1.0 + nb);
        out[1] = nres;
        out[2] = a[P_RESMAX];
        out[3] = a[P_AXMAX];
        out[4] = nb;
        out[5] = a[P_BMAX];
        out[6] = a[P_BLAM];
        out[7] = -a[P_BLAM];
    }
}

}  // namespace

namespace mfs {
// Host side of the checked build's record for the kernels of this file (0 when nothing failed, or in
// the normal build); reset clears it. mfs_debug_bounds reports it when the solver kernels' record is
// empty.
unsigned long long static_bounds_record(bool reset) {
#ifdef MFS_DEBUG_BOUNDS
    unsigned long long v = 0;
    cudaDeviceSynchronize();
    cudaMemcpyFromSymbol(&v, g_bounds_fail, sizeof v);
    if (reset) {
        const unsigned long long zero = 0;
        cudaMemcpyToSymbol(g_bounds_fail, &zero, sizeof zero);
    }
    return v;
#else
    (void)reset;
    return 0;
#endif
}
}  // namespace mfs

extern "C" mfs_status mfs_row_residuals_static(int64_t m, int64_t n, const int32_t* row_ptr, const int32_t* col_idx,
                                               const double* val, const double* b, const double* x,
                                               const double* lambda, double* out, void* cuda_stream) {
    if (!mfs::host::static_resid_args_ok(m, n, (int64_t)RS_MAX_CTAS * RS_ROWS_PER_CTA, row_ptr, col_idx, val, b, x,
                                         lambda, out))
        return MFS_ERR_INVALID;  // includes m beyond the static scratch
    // an error left by earlier work on this thread is reported, not consumed: nothing is enqueued
    if (cudaPeekAtLastError() != cudaSuccess) return MFS_ERR_CUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= RS_MAX_DEVICES) return MFS_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return MFS_ERR_CUDA;
    const CUcontext ctx = current_context();
    double* scratch = nullptr;
    {
        // In host code the array's name is only a stand-in: its device address in the current
        // context is looked up here (set-up), with the device current.
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (cap == cudaStreamCaptureStatusNone) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_row_resid_scratch) != cudaSuccess || !p) return MFS_ERR_CUDA;
            g_scratch_addr[dev] = static_cast<double*>(p);
            g_scratch_ctx[dev] = ctx;
        } else if (!g_scratch_addr[dev] || !ctx || g_scratch_ctx[dev] != ctx) {
            return MFS_ERR_INVALID;  // no call in this context before the capture began
        }
        scratch = g_scratch_addr[dev];
    }
    const int nparts = (int)((m + RS_ROWS_PER_CTA - 1) / RS_ROWS_PER_CTA);
    if (nparts > 0) {
        k_row_resid_static<<<nparts, RS_NT, 0, st>>>((int)m, (int)n, row_ptr, col_idx, val, b, x, lambda, scratch);
        if (cudaGetLastError() != cudaSuccess) return MFS_ERR_CUDA;
    }
    k_row_resid_static_finalize<<<1, RS_NT, 0, st>>>(nparts, scratch, out);
    return cudaGetLastError() == cudaSuccess ? MFS_OK : MFS_ERR_CUDA;
}
