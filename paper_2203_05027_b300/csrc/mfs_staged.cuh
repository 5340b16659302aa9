// mfs_staged.cuh -- the staged FP32 sweeps: the same column and row passes as k_col_sweep /
// k_row_sweep (the reduced form of Algorithm 1, orthant cones), organised so that the gathers read
// shared memory instead of L2.
//
// The gathered vector (v for the column pass, x for the row pass) is cut into blocks of RB entries
// (64 KB in FP32). Each CTA owns a group of consecutive segments (columns or rows, balanced by
// nonzeros, at most a few ten thousand) and keeps one FP32 sum per segment in shared memory. It
// streams every block of the vector into shared memory in turn with bulk asynchronous copies
// (cp.async.bulk, two stages, an mbarrier each) and adds the products of its nonzeros whose
// gathered index falls in that block. The nonzeros of a group are therefore stored sorted by
// block, one 8-byte entry each: the index of the sum it adds to within the group (its "slot") in
// the low 16 bits, the gathered index within the block in the high 16 bits, and the FP32 value.
// Within one (group, block) the entries are cut into NW ranges, one per warp, at segment boundaries
// (precomputed), so that no two warps add into the same segment sum. Within a warp's range the
// entries are laid out in rounds of 32, lane l taking entries l, 32 + l, 64 + l, ... (one coalesced
// 256-byte load per round), and every segment's entries of the block sit in one lane, consecutive
// and in gathered-index order: a lane adds its runs of equal slots in registers and each run's sum
// into shared memory once, with no exchange between lanes. A run longer than a lane holds is cut
// into pieces in several lanes; piece j > 0 of a segment adds into an overflow slot of its own (the
// same one in every block), which the segment's warp folds into the segment's sum, in slot order,
// before its epilogue. Every sum therefore runs in a fixed order (blocks in turn; within a block the
// lane's entries in order), the same on every run.
//
// Every CTA reads the whole vector once per pass (148 x 4 MB for a 10^6-row v), which L2 serves
// at about 25 TB/s to all SMs; the random gathers then cost shared-memory bank cycles instead of
// L2 sector requests. The nonzeros stream from HBM once: the producer warp bulk-prefetches each
// block's entries into L2 a few blocks ahead (marked to leave L2 first, as are the loads that read
// them, so that the vectors the passes read again stay), and every warp loads its entries of the
// next block into registers while it works on the current one. A warp runs the epilogue of its own
// segments as soon as it has seen every block, with its loads batched so that several are in
// flight per thread.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mfs_kernels.cuh"

namespace mfs {
namespace staged {

#ifndef MFS_STG_RB_COL
#define MFS_STG_RB_COL 16384
#define MFS_STG_S_COL 2
#endif
#ifndef MFS_STG_RB_ROW
#define MFS_STG_RB_ROW 16384
#define MFS_STG_S_ROW 2
#endif
#ifndef MFS_STG_ROW_HALVES
#define MFS_STG_ROW_HALVES 2
#endif
#ifndef MFS_STG_ROW_PARTS_MAX
#define MFS_STG_ROW_PARTS_MAX 4
#endif
#ifndef MFS_STG_COL_PARTS_MAX
#define MFS_STG_COL_PARTS_MAX 2
#endif
#ifndef MFS_STG_NW
#define MFS_STG_NW 15
#endif
constexpr int RB_COL = MFS_STG_RB_COL;  // entries of v per block, column pass
constexpr int S_COL = MFS_STG_S_COL;    // stages
constexpr int RB_ROW = MFS_STG_RB_ROW;  // entries of x per block, row pass
constexpr int S_ROW = MFS_STG_S_ROW;
constexpr int ROW_HALVES = MFS_STG_ROW_HALVES;  // row pass: two CTAs per row group, each streaming
                                                // half of x (x is 2.5x longer than v)
constexpr int ROW_PARTS_MAX = MFS_STG_ROW_PARTS_MAX;  // or more parts, where the row groups still fit
                                                      // (fewer, fuller blocks per CTA)
constexpr int COL_PARTS_MAX = MFS_STG_COL_PARTS_MAX;  // column pass: likewise, where v is long enough
                                                      // and the column groups fit (k_col_combine)
constexpr int NW = MFS_STG_NW;  // consumer warps per CTA, plus one producer warp (15: 512 threads, 4 warps
                                // per SM sub-partition, up to 128 registers a thread)
constexpr int NTS = 32 * NW;
constexpr int NTHREADS = NTS + 32;  // the consumer warps and the producer warp
constexpr int MAXG = 24576;    // segments per group (their sums take 96 KB of shared memory)
#ifndef MFS_STG_PFR_COL
#define MFS_STG_PFR_COL 6
#endif
#ifndef MFS_STG_PFR_ROW
#define MFS_STG_PFR_ROW 5
#endif
constexpr int PFR_COL = MFS_STG_PFR_COL;  // rounds of 32 entries a warp prefetches per block (column pass;
                                          // a warp takes about 146 entries of a 64 KB block of v)
constexpr int PFR_ROW = MFS_STG_PFR_ROW;  // (row pass: about 120)
constexpr int PADSEG = 0xFFFF;  // "no slot": a lane with no open run, or no run ending at an entry
constexpr int MAXSLOT = 0x7FFF; // slots (segment sums and overflow sums) per group are below this: an
                                // entry's 16-bit slot is read sign-extended, 0xFFFF being slot -1, the
                                // spare sum in front of the group's sums that padding positions add into
constexpr int EPI_U = 6;       // epilogue items per thread in flight
#ifndef MFS_STG_PDL
#define MFS_STG_PDL 1
#endif
#ifndef MFS_STG_ENT_PD
#define MFS_STG_ENT_PD 2
#endif
#ifndef MFS_STG_KEEP
#define MFS_STG_KEEP 1  // the iterate's vectors read and written by the staged passes carry an L2
                        // evict-last policy (the entries stream past them evict-first)
#endif
#ifndef MFS_STG_ENT_HINT
#define MFS_STG_ENT_HINT 1  // entries loaded with an L2 evict-first policy
#endif
#ifndef MFS_STG_ENT_PF_HINT
#define MFS_STG_ENT_PF_HINT 1  // the producer's L2 prefetch of the entries carries the same policy
#endif

constexpr int ENT_PD = MFS_STG_ENT_PD;  // blocks ahead at which the producer prefetches a block's
                                        // entries into L2 (the consumers load them one block ahead)

// dynamic shared memory of one CTA: the vector stages, the spare sum (16 bytes), the group's sums, its
// split table, 2 S mbarriers
__host__ __device__ constexpr size_t smem_bytes(int rb, int stages, int maxg, int R) {
    return (size_t)stages * rb * 4 + 16 + (size_t)((maxg + 3) / 4 * 4) * 4 + (size_t)((R * (NW + 1) + 3) / 4 * 4) * 4 +
           (size_t)16 * stages;
}

struct StagedArgs {
    const int2* __restrict__ ent;   // entries, sorted by (group, block, segment, gathered index)
    const int* __restrict__ split;  // (G * R) x (NW + 1): warp ranges of each (group, block)
    const int* __restrict__ grp;    // G + 1: first segment of each group
    const int* __restrict__ wseg;   // G x (NW + 1): each warp's first segment within its group
    const int* __restrict__ wovf;   // G x (NW + 1): each warp's first overflow slot within its group
    const int* __restrict__ fold_ptr;  // G * NW + 1: each (group, warp)'s range of fold entries
    const int2* __restrict__ fold;  // (segment, first overflow slot | pieces - 1 << 16), per warp
    const int2* __restrict__ wcone; // column pass with Lorentz cones: G x NW, each warp's cones [x, y)
    // column pass with Lorentz cones: per column 0 orthant, 1 cone fused into this pass, 2 cone left to
    // the big-cone kernel (more than WC columns); per cone 1 if left to the big-cone kernel
    const unsigned char* __restrict__ ctag;
    const unsigned char* __restrict__ soc_big;
    // column pass in parts: k_col_combine's pieces of [0, n), at most CMAXW columns each and never
    // inside a fused cone: first column, end, and the Lorentz cones [z, w) within
    const int4* __restrict__ csub;
    int nsub;
    const float* __restrict__ vec;  // gathered vector, R * rb entries (tail padding unused)
    const float* __restrict__ rinv;  // row pass: 1/(1 + r_i), r_i = sum of a_ik^2 over row i
    const float* __restrict__ dinv;  // column pass: 1/(1 + d_j), d_j = nonzeros of column j
    int* err;                       // set to 1 if a wait for a block gave up
    int G, R, maxg_pad;             // maxg_pad: sum slots (segments and overflow) of the largest group,
                                    // rounded up to a multiple of 4 (padding entries add into slot -1)
    int halves;                     // row pass: CTAs per group, each streaming 1/halves of x (1 or 2)
    float* part;                    // halves > 1: halves x nseg partial row sums
    int nseg;                       // segments of the pass (rows for the row pass)
    int nent;                       // entries (padded), the bound of the checked build
    int spin;                       // polls of an mbarrier before a wait gives up
    int no_loads;                   // diagnostic: issue no copies, so that every wait gives up
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void issue_block(float* dst, const float* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
#if MFS_STG_KEEP
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
#else
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
#endif
}

// Accesses to the iterate's vectors (x, z, delta, c, column pointers; lambda, v, b, row norms, the
// partial row sums) with an L2 evict-last policy when MFS_STG_KEEP is set, plain ones otherwise.
// Evict-last lines stay in the context's persisting L2 set-aside (raised by the solver's set-up), so
// that from one pass to the next the vectors are read from L2 while the entries stream past. The
// accesses are volatile asm (plain accesses in the plain build), so their order among themselves is
// the program's.
__device__ __forceinline__ uint64_t policy_keep() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ float ld_keep(const float* p, uint64_t pol) {
#if MFS_STG_KEEP
    float v;
    asm volatile("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol) : "memory");
    return v;
#else
    return *p;
#endif
}
__device__ __forceinline__ float ldg_keep(const float* p, uint64_t pol) {  // data the pass does not write
#if MFS_STG_KEEP
    float v;
    asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
#else
    return __ldg(p);
#endif
}
__device__ __forceinline__ int ldg_keep(const int* p, uint64_t pol) {
#if MFS_STG_KEEP
    int v;
    asm volatile("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
#else
    return __ldg(p);
#endif
}
// four consecutive floats (p 16-byte aligned), with the policy
__device__ __forceinline__ float4 ld4_keep(const float* p, uint64_t pol) {
    float4 v;
#if MFS_STG_KEEP
    asm volatile("ld.global.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p), "l"(pol)
                 : "memory");
#else
    v = *reinterpret_cast<const float4*>(p);
#endif
    return v;
}
__device__ __forceinline__ void st4_keep(float* p, float4 v, uint64_t pol) {
#if MFS_STG_KEEP
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1,%2,%3,%4}, %5;" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w), "l"(pol)
                 : "memory");
#else
    *reinterpret_cast<float4*>(p) = v;
#endif
}
__device__ __forceinline__ void st_keep(float* p, float v, uint64_t pol) {
#if MFS_STG_KEEP
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol) : "memory");
#else
    *p = v;
#endif
}
// The staged passes' updates multiply by reciprocals computed once (1/mu per launch, 1/(1 + d_j) and
// 1/(1 + r_i) at set-up) instead of dividing: the same steps, FP32 rounding of their own.
// x+ = (d x + A^T v + z + (delta - c)/mu)/(1 + d), written as x + (A^T v + z + (delta - c)/mu - x)/(1 + d)
__device__ __forceinline__ float col_x_step(float x, float atv, float z, float dl, float c, float dinv, float rmu) {
    return x + (atv + z + (dl - c) * rmu - x) * dinv;
}
// the orthant z-step of column j after its x-update, stores with the policy
__device__ __forceinline__ void orthant_keep(const SweepArgs<float>& a, int j, float xn, float dj, float mu,
                                             float rmu, uint64_t pol) {
    st_keep(a.x + j, xn, pol);
    const float w = xn - dj * rmu;
    const float zn = w > 0.f ? w : 0.f;
    st_keep(a.z + j, zn, pol);
    st_keep(a.del + j, dj + mu * (zn - xn), pol);
}
// rho = (b_i - a_i x)/(1 + r_i), lambda and v of row i, stores with the policy
__device__ __forceinline__ void row_keep(const SweepArgs<float>& a, int i, float ax, float rinv, float bi, float li,
                                         float rmu, uint64_t pol) {
    const float rho = (bi - ax) * rinv;
    const float ln = li - a.mu * rho;
    st_keep(a.lam + i, ln, pol);
    st_keep(a.v + i, rho - ln * rmu, pol);
}

// Programmatic dependent launch. The passes are launched so that the next one may start while
// this one runs: each kernel signals that at its start, does only work on data no earlier kernel
// writes (barrier set-up, split table, its first blocks' entries) and then waits until the
// previous kernel has completed and its writes are visible. Every thread waits before its first
// access to the iterate, and every CTA waits before it exits, so a kernel's completion implies
// its predecessor's. Without the launch attribute both instructions return at once.
__device__ __forceinline__ void dep_launch_next() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void dep_wait_prev() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Hint: bring the 16-byte-aligned part of [p, p + bytes) into L2 (a bulk prefetch; no access
// outside the range, no completion to wait for).
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes) {
    const uintptr_t s = ((uintptr_t)p + 15) & ~(uintptr_t)15, e = ((uintptr_t)p + bytes) & ~(uintptr_t)15;
    if (e > s) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(s), "r"((uint32_t)(e - s)) : "memory");
}

// L2 eviction policy of the entries, which are read once: evict first, so that the vectors the
// passes read again stay in L2 while the entries stream past.
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    if (MFS_STG_ENT_HINT)
        asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    else
        asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// prefetch_l2 with an L2 eviction policy for the lines it brings in
__device__ __forceinline__ void prefetch_l2_hint(const void* p, size_t bytes, uint64_t pol) {
    const uintptr_t s = ((uintptr_t)p + 15) & ~(uintptr_t)15, e = ((uintptr_t)p + bytes) & ~(uintptr_t)15;
    if (e > s)
        asm volatile("cp.async.bulk.prefetch.L2.global.L2::cache_hint [%0], %1, %2;" ::"l"(s), "r"((uint32_t)(e - s)),
                     "l"(pol)
                     : "memory");
}

// Bounded wait for phase `parity` of an mbarrier; false if it gave up.
__device__ __forceinline__ bool wait_block(uint64_t* bar, uint32_t parity, int spin) {
    for (int i = 0; i < spin; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Rounds [s0 + 32 r, s0 + 32 r + 32) of a warp's range [s0, s1) for r < PFR: lane l loads entry
// s0 + 32 r + l (one coalesced 256-byte load per round, bypassing L1 and marked first to leave L2:
// each entry is read once); positions at or past s1 hold no entry.
template <int PFR>
__device__ __forceinline__ void load_rounds(const int2* __restrict__ ent, int s0, int s1, int lane, int2 (&e)[PFR],
                                            int nent, uint64_t pol) {
#pragma unroll
    for (int r = 0; r < PFR; ++r) {
        const int q = s0 + r * 32 + lane;
        if (q < s1 && MFS_INB(q, nent, BS_STG_ENT)) {
            asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.b32 {%0,%1}, [%2], %3;"
                : "=r"(e[r].x), "=r"(e[r].y)
                : "l"(ent + q), "l"(pol));
        } else {
            e[r] = make_int2(0xFFFF, 0);  // gathered index 0, value 0, the spare slot -1
        }
    }
}

// PFR consecutive entries of one lane. The lane's open run (slot cur, partial sum) continues while
// the slot repeats; where it changes, the run's sum is added to its slot. Slots that end a run are
// distinct within a lane and owned by that lane in this block, so their read-modify-writes are
// issued as all loads, then all stores.
template <int PFR, int RB>
__device__ __forceinline__ void lane_chunk(const int2 (&e)[PFR], const float* vb, float* acc, int nacc, int& cur,
                                           float& sum) {
    int sg[PFR];
    float p[PFR];
#pragma unroll
    for (int r = 0; r < PFR; ++r) {
        const uint32_t gi = (uint32_t)e[r].x >> 16;
        const int k = (int)(int16_t)(uint16_t)(e[r].x & 0xFFFF);  // padding: -1, the spare slot
#ifdef MFS_DEBUG_BOUNDS
        const bool ok = MFS_INB(gi, RB, BS_STG_VEC) && (k == -1 || MFS_INB(k, nacc, BS_STG_ACC));
        sg[r] = ok ? k : -1;
        p[r] = ok ? __int_as_float(e[r].y) * vb[gi] : 0.f;
#else
        sg[r] = k;
        p[r] = __int_as_float(e[r].y) * vb[gi];
#endif
    }
    int fk[PFR];  // fk[r]: the slot whose run ends just before entry r (PADSEG: none)
    float fv[PFR];
    int c = cur;
    float t = sum;
#pragma unroll
    for (int r = 0; r < PFR; ++r) {
        const bool cont = sg[r] == c;
        fk[r] = cont ? PADSEG : c;
        fv[r] = t;
        t = cont ? t + p[r] : p[r];
        c = sg[r];
    }
    cur = c;
    sum = t;
    float old[PFR];
#pragma unroll
    for (int r = 0; r < PFR; ++r)
        if (fk[r] != PADSEG) old[r] = acc[fk[r]];
#pragma unroll
    for (int r = 0; r < PFR; ++r)
        if (fk[r] != PADSEG) acc[fk[r]] = old[r] + fv[r];
}

// All entries of a warp's range [s0, s1) of one block: the PFR prefetched rounds, then any further
// ones (a range longer than PFR rounds), then the lane's last open run.
template <int PFR, int RB>
__device__ __forceinline__ void run_block(const int2 (&e)[PFR], int s0, int s1, const int2* __restrict__ ent,
                                          const float* vb, float* acc, int lane, int nent, int nacc, uint64_t pol) {
    int cur = PADSEG;
    float sum = 0.f;
    lane_chunk<PFR, RB>(e, vb, acc, nacc, cur, sum);
    for (int b0 = s0 + PFR * 32; b0 < s1; b0 += PFR * 32) {
        int2 t[PFR];
        load_rounds<PFR>(ent, b0, s1, lane, t, nent, pol);
        lane_chunk<PFR, RB>(t, vb, acc, nacc, cur, sum);
    }
    if (cur != PADSEG) acc[cur] += sum;
}

// Block u of the CTA's sequence of staged blocks sits in stage u % S; full[k] completes when its
// copy has landed, empty[k] when every consumer warp has finished with it.
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// The producer's L2 prefetch of all warps' entries of block b (one contiguous range per block)
__device__ __forceinline__ void prefetch_entries(const StagedArgs& g, const int* spl, int b, uint64_t pol) {
    const int e0 = spl[b * (NW + 1)], e1 = spl[b * (NW + 1) + NW];
    if (MFS_STG_ENT_PF_HINT)
        prefetch_l2_hint(g.ent + e0, (size_t)(e1 - e0) * sizeof(int2), pol);
    else
        prefetch_l2(g.ent + e0, (size_t)(e1 - e0) * sizeof(int2));
}

// Consumer side of block b (the CTA's block u): load the warp's entries of block b + 1 into D (the
// producer has prefetched them into L2), wait for the stage, add the entries held in C, and
// release the stage.
template <int RB, int PFR, int S>
__device__ __forceinline__ void block_step(int b, int be, uint32_t u, int2 (&C)[PFR], int2 (&D)[PFR], const int* spl,
                                           const StagedArgs& g, const float* vb, float* acc, uint64_t* full,
                                           uint64_t* empty, bool& bad, int warp, int lane, uint64_t pol) {
    if (b + 1 < be) {
        const int* sp = spl + (b + 1) * (NW + 1) + warp;
        load_rounds<PFR>(g.ent, sp[0], sp[1], lane, D, g.nent, pol);
    }
    const uint32_t k = u % S;
    if (!wait_block(full + k, (u / S) & 1u, g.spin)) bad = true;
    const int* sp = spl + b * (NW + 1) + warp;
    run_block<PFR, RB>(C, sp[0], sp[1], g.ent, vb + k * RB, acc, lane, g.nent, g.maxg_pad, pol);
    __syncwarp();
    if (lane == 0) mbar_arrive(empty + k);
}

// The column pass's epilogue of the columns k0 + [ws, we) (one warp): x+ from the sums (Algorithm 1,
// the x-step in reduced form), the orthant z-step and delta-update, and the Lorentz cones wc.x ..
// wc.y - 1, which lie within these columns (eq. proj). acc[t] holds A^T v of column k0 + t for t in
// [ws, we) (with PARTS: the parts' sums in g.part, added in a fixed order as they are loaded, acc
// only receiving w); for the fused cones' columns it is overwritten by w = x+ - delta/mu.
template <bool SOC, bool PARTS>
__device__ __forceinline__ void col_epilogue(const StagedArgs& g, const SweepArgs<float>& a, float* acc, int k0,
                                             int ws, int we, int2 wc, int lane) {
    const int e0 = ws + lane, e1 = we, es = 32;
    const float mu = a.mu, rmu = 1.f / mu;
    const uint64_t kp = policy_keep();
    for (int t0 = e0; t0 < e1; t0 += es * EPI_U) {
        float px[EPI_U], pz[EPI_U], pd[EPI_U], pc[EPI_U], dg[EPI_U], pa[EPI_U];
        int tag[EPI_U];
#pragma unroll
        for (int q = 0; q < EPI_U; ++q) {
            const int t = t0 + q * es;
            if (t < e1) {
                const int j = k0 + t;
                dg[q] = ldg_keep(g.dinv + j, kp);
                px[q] = ld_keep(a.x + j, kp);
                pz[q] = ld_keep(a.z + j, kp);
                pd[q] = ld_keep(a.del + j, kp);
                pc[q] = ldg_keep(a.c + j, kp);
                tag[q] = SOC ? __ldg(g.ctag + j) : 0;
                if (PARTS) {
                    float v = ld_keep(g.part + j, kp);
                    for (int h = 1; h < g.halves; ++h) v += ld_keep(g.part + (size_t)h * g.nseg + j, kp);
                    pa[q] = v;
                }
            }
        }
#pragma unroll
        for (int q = 0; q < EPI_U; ++q) {
            const int t = t0 + q * es;
            if (t < e1) {
                const float xn = col_x_step(px[q], PARTS ? pa[q] : acc[t], pz[q], pd[q], pc[q], dg[q], rmu);
                if (!SOC || tag[q] == 0) {
                    orthant_keep(a, k0 + t, xn, pd[q], mu, rmu, kp);
                } else {
                    st_keep(a.x + k0 + t, xn, kp);  // a cone too large to fuse: the big-cone kernel follows
                    if (tag[q] == 1) acc[t] = xn - pd[q] * rmu;  // w of the z-step, kept in place
                }
            }
        }
    }
    if (SOC) {
        // The Lorentz cones wc.x .. wc.y - 1 (never straddling warps; acc holds w = x+ - delta/mu of
        // the fused ones' columns): their descriptors loaded 32 at a time, one per lane, then four
        // cones at a time, eight lanes each: ||w_tail||^2 by strided sums and three shuffles, then
        // the z-step (eq. proj) over the cone's columns and delta+ = delta + mu (z+ - x+) = mu (z+ - w).
        // Cones too large to fuse keep their columns for the big-cone kernel.
        __syncwarp();
        const int r = lane & 7, u = lane >> 3;
        for (int q0 = wc.x; q0 < wc.y; q0 += 32) {
            const int q = q0 + lane;
            int st = 0, sz = 0;  // this lane's cone: first column (from k0), size (0: none or not fused)
            if (q < wc.y && !g.soc_big[q]) {
                st = a.soc_start[q] - k0;
                sz = a.soc_size[q];
            }
            const int nb = (min(32, wc.y - q0) + 3) >> 2;
            for (int bq = 0; bq < nb; ++bq) {
                const int cs = __shfl_sync(FULL, st, 4 * bq + u), cz = __shfl_sync(FULL, sz, 4 * bq + u);
                float ss = 0.f;
                for (int t = 1 + r; t < cz; t += 8) ss += acc[cs + t] * acc[cs + t];
                ss += __shfl_xor_sync(FULL, ss, 1);
                ss += __shfl_xor_sync(FULL, ss, 2);
                ss += __shfl_xor_sync(FULL, ss, 4);
                const float alpha = sqrtf(ss), w1 = cz > 0 ? acc[cs] : 0.f;
                const float ia = alpha > 0.f ? 0.5f / alpha : 0.f;  // (used only where alpha > |w1|)
                for (int t = r; t < cz; t += 8) {
                    const float w = acc[cs + t];
                    // eq. proj: 0 below the polar cone, w inside K, else the boundary point
                    const float zt = alpha <= -w1 ? 0.f
                                     : alpha <= w1 ? w
                                     : (t == 0 ? 0.5f * (w + alpha) : 0.5f * w + w1 * w * ia);
                    st_keep(a.z + k0 + cs + t, zt, kp);
                    st_keep(a.del + k0 + cs + t, mu * (zt - w), kp);
                }
            }
        }
    }
}

// MODE 0: column pass (gathers v; epilogue x-, z-, delta-updates; with SOC also the z-step of the
// small Lorentz cones, whose columns never straddle two warps' ranges).
// MODE 1: row pass (gathers x; epilogue rho, lambda and v of each row).
// Warps 0..NW-1 consume; warp NW produces (its lane 0 issues the copies of the vector blocks).
// Warp w owns the segments wseg[w] .. wseg[w+1]-1 of its group in every block: it alone adds into
// their sums, and it runs their epilogue as soon as it has seen every block, while other warps
// may still be streaming.
template <int MODE, int RB, int PFR, int S, bool SOC>
__global__ void __launch_bounds__(NTHREADS, 1) k_staged(const StagedArgs g, const SweepArgs<float> a) {
    extern __shared__ __align__(128) unsigned char smem[];
    float* vb = reinterpret_cast<float*>(smem);
    float* acc = vb + S * RB + 4;  // acc[-1]: the spare sum of the padding positions
    const int R = g.R;
    int* spl = reinterpret_cast<int*>(acc + g.maxg_pad);
    uint64_t* full = reinterpret_cast<uint64_t*>(spl + (R * (NW + 1) + 3) / 4 * 4);
    uint64_t* empty = full + S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    dep_launch_next();
    if (threadIdx.x == 0) {
        for (int k = 0; k < S; ++k) {
            mbar_init(full + k, 1);
            mbar_init(empty + k, NW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t u0 = 0;  // the CTA's staged blocks before the current group
    bool bad = false;
    const int H = g.halves;
    for (int part = blockIdx.x; part < g.G * H; part += gridDim.x) {
        // group grp; this CTA streams blocks [bb, be) of the vector (all of them unless H > 1)
        const int grp = part / H, h = part % H;
        const int bb = (int)((long long)R * h / H), be = (int)((long long)R * (h + 1) / H);
        const int k0 = g.grp[grp];
        const int* gs = g.split + (size_t)grp * R * (NW + 1);
        for (int t = threadIdx.x; t < R * (NW + 1); t += NTHREADS) spl[t] = gs[t];
        __syncthreads();  // split table in place; the previous group's sums are no longer read
        if (warp == NW) {
            dep_wait_prev();  // the vector was written by the previous pass
            if (lane == 0 && !g.no_loads) {
                const uint64_t epol = policy_evict_first();
                for (int b = bb; b < be && b < bb + ENT_PD; ++b) prefetch_entries(g, spl, b, epol);
                for (int b = bb; b < be; ++b) {
                    const uint32_t u = u0 + (b - bb), k = u % S;
                    if (u >= S && !wait_block(empty + k, (u / S - 1) & 1u, g.spin)) bad = true;
                    issue_block(vb + k * RB, g.vec + (size_t)b * RB, RB * 4u, full + k);
                    if (b + ENT_PD < be) prefetch_entries(g, spl, b + ENT_PD, epol);
                }
            }
        } else {
            const int ws = g.wseg[grp * (NW + 1) + warp], we = g.wseg[grp * (NW + 1) + warp + 1];
            const int os = g.wovf[grp * (NW + 1) + warp], oe = g.wovf[grp * (NW + 1) + warp + 1];
            for (int t = ws + lane; t < we; t += 32) acc[t] = 0.f;
            for (int t = os + lane; t < oe; t += 32) acc[t] = 0.f;
            __syncwarp();
            const uint64_t pol = policy_evict_first();
            int2 A[PFR], B[PFR];
            if (bb < be)
                load_rounds<PFR>(g.ent, spl[bb * (NW + 1) + warp], spl[bb * (NW + 1) + warp + 1], lane, A, g.nent, pol);
            dep_wait_prev();  // the epilogue reads and writes the iterate
            for (int b = bb; b < be; b += 2) {
                const uint32_t u = u0 + (b - bb);
                block_step<RB, PFR, S>(b, be, u, A, B, spl, g, vb, acc, full, empty, bad, warp, lane, pol);
                if (b + 1 < be)
                    block_step<RB, PFR, S>(b + 1, be, u + 1, B, A, spl, g, vb, acc, full, empty, bad, warp, lane, pol);
            }
            __syncwarp();
            // pieces of long runs: each segment's overflow sums added to it in slot order
            for (int f = g.fold_ptr[grp * NW + warp] + lane; f < g.fold_ptr[grp * NW + warp + 1]; f += 32) {
                const int2 fd = g.fold[f];
                const int k0 = fd.y & 0xFFFF, cnt = fd.y >> 16;
                float v = acc[fd.x];
                for (int j = 0; j < cnt; ++j) v += acc[k0 + j];
                acc[fd.x] = v;
            }
            __syncwarp();
            // the epilogue of the warp's own segments, as soon as the warp has seen every block
            const int e0 = ws + lane, e1 = we, es = 32;
            if (H > 1) {  // partial sums; k_col_combine / k_row_combine add the parts
                const uint64_t kp = policy_keep();
                float* out = g.part + (size_t)h * g.nseg + k0;
                for (int t = e0; t < e1; t += es) st_keep(out + t, acc[t], kp);
            } else if (MODE == 0) {
                col_epilogue<SOC, false>(g, a, acc, k0, ws, we, SOC ? g.wcone[grp * NW + warp] : make_int2(0, 0),
                                         lane);
            } else {
                const uint64_t kp = policy_keep();
                const float rmu = 1.f / a.mu;
                for (int t0 = e0; t0 < e1; t0 += es * EPI_U) {
                    float pr[EPI_U], pb[EPI_U], pl[EPI_U];
#pragma unroll
                    for (int q = 0; q < EPI_U; ++q) {
                        const int t = t0 + q * es;
                        if (t < e1) {
                            const int i = k0 + t;
                            pr[q] = ldg_keep(g.rinv + i, kp);
                            pb[q] = ldg_keep(a.b + i, kp);
                            pl[q] = ld_keep(a.lam + i, kp);
                        }
                    }
#pragma unroll
                    for (int q = 0; q < EPI_U; ++q) {
                        const int t = t0 + q * es;
                        if (t < e1) row_keep(a, k0 + t, acc[t], pr[q], pb[q], pl[q], rmu, kp);
                    }
                }
            }
        }
        u0 += (uint32_t)(be - bb);
        __syncthreads();  // the group is done: its sums and split table may be replaced
    }
    dep_wait_prev();  // (a CTA without a group)
    if (bad) {
        // a copy may still be in flight into a stage: wait (bounded) for the last load of each stage
        for (int d = 1; d <= S && (uint32_t)d <= u0; ++d) {
            const uint32_t u = u0 - d;
            wait_block(full + u % S, (u / S) & 1u, g.spin);
        }
        atomicExch(g.err, 1);
    }
}

// Row pass with halves > 1: the partial sums of each row, added in a fixed order (part 0 first),
// then rho, lambda and v (as the row pass's own epilogue).
__global__ void __launch_bounds__(256) k_row_combine(const StagedArgs g, const SweepArgs<float> a) {
    dep_launch_next();
    dep_wait_prev();
    const int m = g.nseg;
    const uint64_t kp = policy_keep();
    const float rmu = 1.f / a.mu, mu = a.mu;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    // four rows at a time with 16-byte accesses where every array allows it (m a multiple of 4, so
    // that each part starts aligned too), the same arithmetic row by row as below
    const bool vec = (m & 3) == 0 && (((uintptr_t)g.part | (uintptr_t)g.rinv | (uintptr_t)a.b | (uintptr_t)a.lam |
                                        (uintptr_t)a.v) & 15) == 0;
    const int m4 = vec ? m / 4 : 0;
    for (int q = tid; q < m4; q += nth) {
        const int i = 4 * q;
        float4 ax = ld4_keep(g.part + i, kp);
        for (int h = 1; h < g.halves; ++h) {
            const float4 p = ld4_keep(g.part + (size_t)h * m + i, kp);
            ax.x += p.x;
            ax.y += p.y;
            ax.z += p.z;
            ax.w += p.w;
        }
        const float4 r = ld4_keep(g.rinv + i, kp), bi = ld4_keep(a.b + i, kp), li = ld4_keep(a.lam + i, kp);
        float4 ln, vn;
        float rho;
        rho = (bi.x - ax.x) * r.x;
        ln.x = li.x - mu * rho;
        vn.x = rho - ln.x * rmu;
        rho = (bi.y - ax.y) * r.y;
        ln.y = li.y - mu * rho;
        vn.y = rho - ln.y * rmu;
        rho = (bi.z - ax.z) * r.z;
        ln.z = li.z - mu * rho;
        vn.z = rho - ln.z * rmu;
        rho = (bi.w - ax.w) * r.w;
        ln.w = li.w - mu * rho;
        vn.w = rho - ln.w * rmu;
        st4_keep(a.lam + i, ln, kp);
        st4_keep(a.v + i, vn, kp);
    }
    for (int i = 4 * m4 + tid; i < m; i += nth) {
        float ax = ld_keep(g.part + i, kp);
        for (int h = 1; h < g.halves; ++h) ax += ld_keep(g.part + (size_t)h * m + i, kp);
        row_keep(a, i, ax, ldg_keep(g.rinv + i, kp), ldg_keep(a.b + i, kp), ld_keep(a.lam + i, kp), rmu, kp);
    }
}

// Column pass in parts (halves > 1): the parts' sums of each column added in a fixed order (part 0
// first), then the column epilogue, cones included, by one warp per piece of at most CMAXW columns
// (the pieces never cut a fused cone), its sums held in shared memory.
constexpr int CSUB = 128;             // target columns per piece
constexpr int CMAXW = CSUB + 64;      // at most (a cut moves to the end of a cone of <= 64 columns)
constexpr int CWPB = 8;               // warps per CTA
template <bool SOC>
__global__ void __launch_bounds__(32 * CWPB, 3) k_col_combine(const StagedArgs g, const SweepArgs<float> a) {
    __shared__ float cbuf[CWPB][CMAXW];
    dep_launch_next();
    dep_wait_prev();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = blockIdx.x * CWPB + warp;
    if (p >= g.nsub) return;  // (no block-wide barrier follows)
    const int4 d = g.csub[p];
    if (!MFS_INB(d.y - d.x - 1, CMAXW, BS_STG_ACC)) return;
    float* acc = &cbuf[warp][0] - d.x;  // w of the fused cones' columns j in [d.x, d.y)
    col_epilogue<SOC, true>(g, a, acc, 0, d.x, d.y, make_int2(d.z, d.w), lane);
}

// the two instantiations the solver launches
#define MFS_STAGED_COL \
    ::mfs::staged::k_staged<0, ::mfs::staged::RB_COL, ::mfs::staged::PFR_COL, ::mfs::staged::S_COL, false>
#define MFS_STAGED_COL_SOC \
    ::mfs::staged::k_staged<0, ::mfs::staged::RB_COL, ::mfs::staged::PFR_COL, ::mfs::staged::S_COL, true>
#define MFS_COL_COMBINE ::mfs::staged::k_col_combine<false>
#define MFS_COL_COMBINE_SOC ::mfs::staged::k_col_combine<true>
#define MFS_STAGED_ROW \
    ::mfs::staged::k_staged<1, ::mfs::staged::RB_ROW, ::mfs::staged::PFR_ROW, ::mfs::staged::S_ROW, false>

}  // namespace staged
}  // namespace mfs
