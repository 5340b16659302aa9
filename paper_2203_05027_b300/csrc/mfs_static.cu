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
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/mfs.h"

namespace {

constexpr int RS_NT = 256;                      // threads per CTA
constexpr int RS_ROWS_PER_CTA = 256;            // rows per CTA (one warp takes every 8th row)
constexpr int RS_MAX_CTAS = 16384;              // scratch rows
constexpr int RS_NPART = 8;                     // doubles per scratch row (6 used)
constexpr int RS_MAX_DEVICES = 64;

enum : int { P_RES2 = 0, P_RESMAX, P_AXMAX, P_B2, P_BMAX, P_BLAM };

static __device__ __align__(256) double g_row_resid_scratch[RS_MAX_CTAS * RS_NPART];

std::mutex g_setup_mutex;
double* g_scratch_addr[RS_MAX_DEVICES] = {};  // device address of the array, per device

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    return v;
}

// Per-CTA partials: sum (Ax-b)^2, max |Ax-b|, max |Ax|, sum b^2, max |b|, sum b*lambda over the
// CTA's rows, FP64, one warp per row, fixed order (deterministic).
__global__ void __launch_bounds__(RS_NT) k_row_resid_static(int m, const int* __restrict__ row_ptr,
                                                            const int* __restrict__ col_idx,
                                                            const double* __restrict__ val,
                                                            const double* __restrict__ b,
                                                            const double* __restrict__ x,
                                                            const double* __restrict__ lam, double* scratch) {
    __shared__ double sh[RS_NT / 32][6];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r0 = blockIdx.x * RS_ROWS_PER_CTA;
    double f[6] = {0, 0, 0, 0, 0, 0};
    for (int rl = warp; rl < RS_ROWS_PER_CTA; rl += RS_NT / 32) {
        const int i = r0 + rl;
        if (i >= m) break;
        double ax = 0.0;
        for (int k = row_ptr[i] + lane; k < row_ptr[i + 1]; k += 32) ax += val[k] * x[col_idx[k]];
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

extern "C" mfs_status mfs_row_residuals_static(int64_t m, int64_t n, const int32_t* row_ptr, const int32_t* col_idx,
                                               const double* val, const double* b, const double* x,
                                               const double* lambda, double* out, void* cuda_stream) {
    if (m < 0 || n < 0) return MFS_ERR_INVALID;
    if (m > (int64_t)RS_MAX_CTAS * RS_ROWS_PER_CTA) return MFS_ERR_INVALID;  // beyond the static scratch
    if (!out || (m && (!row_ptr || !b || !lambda)) || (n && !x)) return MFS_ERR_INVALID;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= RS_MAX_DEVICES) return MFS_ERR_CUDA;
    double* scratch = nullptr;
    {
        // Set-up, once per device, with that device current: in host code the array's name is
        // only a stand-in, so its device address is looked up here and kept.
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_row_resid_scratch) != cudaSuccess || !p) return MFS_ERR_CUDA;
            g_scratch_addr[dev] = static_cast<double*>(p);
        }
        scratch = g_scratch_addr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int nparts = (int)((m + RS_ROWS_PER_CTA - 1) / RS_ROWS_PER_CTA);
    if (nparts > 0)
        k_row_resid_static<<<nparts, RS_NT, 0, st>>>((int)m, row_ptr, col_idx, val, b, x, lambda, scratch);
    k_row_resid_static_finalize<<<1, RS_NT, 0, st>>>(nparts, scratch, out);
    return cudaGetLastError() == cudaSuccess ? MFS_OK : MFS_ERR_CUDA;
}
