// mfs_device.cuh -- device building blocks for the sm_103a sweep kernels: 256-bit global loads,
// the warp-level segmented scan that turns per-nonzero products into per-column (or per-row)
// sums, and deterministic reductions.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mfs {

constexpr int NT = 256;           // threads per CTA
constexpr int NWARP = NT / 32;    // warps per CTA; each warp owns one chunk
constexpr int IPT = 8;            // consecutive nonzeros held by one lane
constexpr int WT = 32 * IPT;      // nonzeros per chunk (a longer single column/row is a "long" chunk)
constexpr int WC = 64;            // columns (or rows) per chunk
constexpr int CPL = WC / 32;      // columns (or rows) per lane in a chunk epilogue
constexpr int PAD = 8;            // chunk starts in the padded nonzero arrays are multiples of 8
constexpr int TAIL = WT;          // the padded nonzero arrays end with this many spare entries
constexpr unsigned FULL = 0xffffffffu;

// Bounds-checked build (-DMFS_DEBUG_BOUNDS, libmfs_bounds.so): every gather index, padded-entry
// load and shared-memory index of the single-instance sweep and residual kernels is checked; a
// failed check records its site and index (the first one wins) and the access is skipped (the value
// read as 0) instead of trapping. A stand-in for a memory checker. In the normal build the checks
// compile to nothing.
enum BoundsSite : int {
    BS_ENTRIES = 1,   // padded nonzero arrays of the chunked layout
    BS_GATHER_V = 2,  // v gathered by the column sweep
    BS_GATHER_X = 3,  // x gathered by the row sweep
    BS_GATHER_L = 4,  // lambda gathered by the column residual
    BS_GATHER_XR = 5, // x gathered by the row residual
    BS_STG_VEC = 6,   // staged vector block in shared memory
    BS_STG_ACC = 7,   // staged segment sums in shared memory
    BS_STG_ENT = 8,   // staged entry arrays
    BS_STATIC_ENT = 9,  // mfs_row_residuals_static: nonzero index beyond row_ptr[m]
    BS_STATIC_X = 10    // mfs_row_residuals_static: column index outside [0, n)
};
#ifdef MFS_DEBUG_BOUNDS
static __device__ unsigned long long g_bounds_fail;  // (site << 40) | low 40 bits of the index
__device__ __forceinline__ bool in_bounds(long long idx, long long lim, int site) {
    const bool ok = idx >= 0 && idx < lim;
    if (!ok) atomicCAS(&g_bounds_fail, 0ull, ((unsigned long long)site << 40) | ((unsigned long long)idx & 0xFFFFFFFFFFull));
    return ok;
}
#define MFS_INB(idx, lim, site) ::mfs::in_bounds((long long)(idx), (long long)(lim), (site))
#else
#define MFS_INB(idx, lim, site) true
#endif

// Shared-memory slot of local nonzero e in a per-warp array: one word of padding per 32 keeps
// the lanes' segment-end stores (lane l writes near 8l) off the same banks.
__device__ __forceinline__ int eslot(int e) {
    return e + (e >> 5);
}
constexpr int ESLOTS = WT + WT / 32;

// Eight consecutive 32-bit (or four 64-bit) elements in one 256-bit load; read-only data that is
// streamed once per sweep, so it bypasses L1. The address must be 32-byte aligned.
__device__ __forceinline__ void ld256(const int* p, int (&o)[8]) {
    asm volatile("ld.global.nc.L1::no_allocate.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(o[0]), "=r"(o[1]), "=r"(o[2]), "=r"(o[3]), "=r"(o[4]), "=r"(o[5]), "=r"(o[6]), "=r"(o[7])
                 : "l"(p));
}
__device__ __forceinline__ void ld256(const float* p, float (&o)[8]) {
    asm volatile("ld.global.nc.L1::no_allocate.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(o[0]), "=f"(o[1]), "=f"(o[2]), "=f"(o[3]), "=f"(o[4]), "=f"(o[5]), "=f"(o[6]), "=f"(o[7])
                 : "l"(p));
}
__device__ __forceinline__ void ld256(const double* p, double (&o)[8]) {
    asm volatile("ld.global.nc.L1::no_allocate.v4.f64 {%0,%1,%2,%3}, [%4];"
                 : "=d"(o[0]), "=d"(o[1]), "=d"(o[2]), "=d"(o[3])
                 : "l"(p));
    asm volatile("ld.global.nc.L1::no_allocate.v4.f64 {%0,%1,%2,%3}, [%4];"
                 : "=d"(o[4]), "=d"(o[5]), "=d"(o[6]), "=d"(o[7])
                 : "l"(p + 4));
}

// Unevaluated sum hi + lo of two floats, used to accumulate FP32 data with about twice FP32's
// precision (B300 runs FP64 at a small fraction of its FP32 rate). The error-free transformations
// are Knuth's TwoSum and the FMA form of Dekker's TwoProduct; the sum of two pairs adds the
// low parts into the rounding error of the high parts and renormalises (fast TwoSum).
struct DF {
    float hi, lo;
    DF() = default;
    __device__ __forceinline__ explicit DF(int) : hi(0.f), lo(0.f) {}
    __device__ __forceinline__ DF(float h, float l) : hi(h), lo(l) {}
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ DF df_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return DF(p, __fmaf_rn(a, b, -p));
}

__device__ __forceinline__ DF operator+(const DF& a, const DF& b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float h = __fadd_rn(s, e);
    return DF(h, __fsub_rn(e, __fsub_rn(h, s)));
}

__device__ __forceinline__ double to_double(const DF& a) {
    return double(a.hi) + double(a.lo);
}
__device__ __forceinline__ double to_double(double a) {
    return a;
}
__device__ __forceinline__ double to_double(float a) {
    return double(a);
}
// pair helpers for reductions: maxima compare normalised pairs (hi first, then lo)
__device__ __forceinline__ DF df_from(double d) {
    const float h = (float)d;
    return DF(h, (float)(d - (double)h));
}
__device__ __forceinline__ DF df_neg(const DF& a) {
    return DF(-a.hi, -a.lo);
}
__device__ __forceinline__ DF df_abs(const DF& a) {
    return a.hi < 0.f ? df_neg(a) : a;
}
__device__ __forceinline__ DF df_sq(const DF& a) {  // a^2, dropping lo^2 (relative 2^-48)
    const float p = __fmul_rn(a.hi, a.hi);
    return DF(p, __fmaf_rn(__fmul_rn(2.f, a.hi), a.lo, __fmaf_rn(a.hi, a.hi, -p)));
}
__device__ __forceinline__ DF df_max(const DF& a, const DF& b) {
    return (a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo)) ? a : b;
}

__device__ __forceinline__ float shfl_up(float v, int d) {
    return __shfl_up_sync(FULL, v, d);
}
__device__ __forceinline__ double shfl_up(double v, int d) {
    return __shfl_up_sync(FULL, v, d);
}
__device__ __forceinline__ DF shfl_up(const DF& v, int d) {
    return DF(__shfl_up_sync(FULL, v.hi, d), __shfl_up_sync(FULL, v.lo, d));
}

template <typename A, int NV>
struct Sums {
    A v[NV];
};

// Warp-wide exclusive segmented scan in lane order. Each lane brings (flag = "a segment starts
// among my items", val = sum of my items after my last segment start, or of all of them if none
// starts) and gets the sum of the segment still open when its items begin (its carry-in).
template <typename A, int NV>
__device__ __forceinline__ Sums<A, NV> warp_seg_carry(bool flag, const Sums<A, NV>& val) {
    const int lane = threadIdx.x & 31;
    int f = flag ? 1 : 0;
    Sums<A, NV> s = val;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int fu = __shfl_up_sync(FULL, f, d);
        Sums<A, NV> su;
#pragma unroll
        for (int t = 0; t < NV; ++t) su.v[t] = shfl_up(s.v[t], d);
        if (lane >= d) {
            if (!f) {
#pragma unroll
                for (int t = 0; t < NV; ++t) s.v[t] = su.v[t] + s.v[t];
            }
            f |= fu;
        }
    }
    Sums<A, NV> out;
#pragma unroll
    for (int t = 0; t < NV; ++t) {
        out.v[t] = shfl_up(s.v[t], 1);
        if (lane == 0) out.v[t] = A(0);
    }
    return out;
}

// Deterministic block reduction (sum) of NV values; result valid in thread 0.
// sh needs NWARP*NV elements. Two __syncthreads.
template <typename A, int NV>
__device__ __forceinline__ Sums<A, NV> block_sum(Sums<A, NV> s, A* sh) {
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

}  // namespace mfs
