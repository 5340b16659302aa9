// mfs_device.cuh -- device building blocks for the sm_103a sweep kernels:
// bulk (TMA 1-D) copies into shared memory on an mbarrier with bounded waits, and the block-wide
// segmented scan that turns per-nonzero products into per-column (or per-row) sums.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mfs {

constexpr int NT = 256;              // threads per CTA of the sweep kernels
constexpr int NWARP = NT / 32;
constexpr int IPT = 8;               // consecutive nonzeros owned by one thread
constexpr int TILE = NT * IPT;       // nonzeros per chunk (a longer single column/row loops)
constexpr int CMAX = 1024;           // columns (or rows) per chunk
constexpr int CPT = CMAX / NT;       // columns per thread in a chunk epilogue
constexpr int PAD = 8;               // chunk starts in the padded nonzero arrays are multiples of 8

// error codes written to the device error word
constexpr int DERR_TIMEOUT = 1;

// Spin limit of a bounded mbarrier wait. Each try_wait may itself suspend for a while, so this is
// generous; a wait that runs out records DERR_TIMEOUT and the CTA returns.
constexpr uint32_t MBAR_SPIN_LIMIT = 1u << 22;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// 1-D bulk copy global -> shared, completing on the mbarrier. Both addresses 16-byte aligned,
// bytes a multiple of 16 (the chunked layout guarantees 32-byte alignment of every chunk).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Thread 0 waits (bounded) for phase `parity` of the barrier; the verdict is broadcast through
// shared memory so that every thread of the CTA takes the same branch. On a timeout the error
// word gets DERR_TIMEOUT, the copy gets one more bounded chance to land, and false is returned.
__device__ __forceinline__ bool cta_wait_bulk(uint64_t* bar, uint32_t parity, int* s_ok, int* err) {
    if (threadIdx.x == 0) {
        bool done = false;
        for (uint32_t i = 0; i < MBAR_SPIN_LIMIT && !done; ++i) done = mbar_try_wait(bar, parity);
        if (!done) {
            atomicCAS(err, 0, DERR_TIMEOUT);
            for (uint32_t i = 0; i < MBAR_SPIN_LIMIT; ++i)
                if (mbar_try_wait(bar, parity)) break;
        }
        *s_ok = done ? 1 : 0;
    }
    __syncthreads();
    return *s_ok != 0;
}

template <typename A, int NV>
struct Sums {
    A v[NV];
};

// Block-wide exclusive segmented scan over the NT threads, in thread order. Each thread brings
// (flag = "a segment starts among my items", val = sum of my items after my last segment start,
// or of all of them if none starts). Returns, per thread, the sum of the segment that is still
// open when its items begin (the carry-in). Deterministic: fixed combination order.
// sh_val needs NWARP*NV elements, sh_flag NWARP ints. Contains one __syncthreads.
template <typename A, int NV>
__device__ __forceinline__ Sums<A, NV> block_seg_carry(bool flag, const Sums<A, NV>& val, A* sh_val,
                                                       int* sh_flag) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    int f = flag ? 1 : 0;
    Sums<A, NV> s = val;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int fu = __shfl_up_sync(FULL, f, d);
        Sums<A, NV> su;
#pragma unroll
        for (int t = 0; t < NV; ++t) su.v[t] = __shfl_up_sync(FULL, s.v[t], d);
        if (lane >= d) {
            if (!f) {
#pragma unroll
                for (int t = 0; t < NV; ++t) s.v[t] = su.v[t] + s.v[t];
            }
            f |= fu;
        }
    }
    // exclusive within the warp
    int fe = __shfl_up_sync(FULL, f, 1);
    Sums<A, NV> se;
#pragma unroll
    for (int t = 0; t < NV; ++t) se.v[t] = __shfl_up_sync(FULL, s.v[t], 1);
    if (lane == 0) {
        fe = 0;
#pragma unroll
        for (int t = 0; t < NV; ++t) se.v[t] = A(0);
    }
    if (lane == 31) {
        sh_flag[warp] = f;
#pragma unroll
        for (int t = 0; t < NV; ++t) sh_val[warp * NV + t] = s.v[t];
    }
    __syncthreads();
    Sums<A, NV> pv;
#pragma unroll
    for (int t = 0; t < NV; ++t) pv.v[t] = A(0);
    for (int w = 0; w < warp; ++w) {
        if (sh_flag[w]) {
#pragma unroll
            for (int t = 0; t < NV; ++t) pv.v[t] = sh_val[w * NV + t];
        } else {
#pragma unroll
            for (int t = 0; t < NV; ++t) pv.v[t] = pv.v[t] + sh_val[w * NV + t];
        }
    }
    Sums<A, NV> out;
#pragma unroll
    for (int t = 0; t < NV; ++t) out.v[t] = fe ? se.v[t] : pv.v[t] + se.v[t];
    return out;
}

// Deterministic block reduction (sum) of NV values; result valid in thread 0.
// sh needs NWARP*NV elements. Contains one __syncthreads (plus one on entry for reuse safety).
template <typename A, int NV>
__device__ __forceinline__ Sums<A, NV> block_sum(Sums<A, NV> s, A* sh) {
    const unsigned FULL = 0xffffffffu;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1)
#pragma unroll
        for (int t = 0; t < NV; ++t) s.v[t] = s.v[t] + __shfl_down_sync(FULL, s.v[t], d);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int t = 0; t < NV; ++t) sh[warp * NV + t] = s.v[t];
    __syncthreads();
    Sums<A, NV> out;
#pragma unroll
    for (int t = 0; t < NV; ++t) out.v[t] = A(0);
    if (threadIdx.x == 0)
        for (int w = 0; w < NWARP; ++w)
#pragma unroll
            for (int t = 0; t < NV; ++t) out.v[t] = out.v[t] + sh[w * NV + t];
    return out;
}

// Deterministic block max of one double; result valid in thread 0.
__device__ __forceinline__ double block_max(double s, double* sh) {
    const unsigned FULL = 0xffffffffu;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s = fmax(s, __shfl_down_sync(FULL, s, d));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = s;
    __syncthreads();
    double out = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < NWARP; ++w) out = fmax(out, sh[w]);
    return out;
}

}  // namespace mfs
