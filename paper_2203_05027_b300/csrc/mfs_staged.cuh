// mfs_staged.cuh -- the staged FP32 sweeps: the same column and row passes as k_col_sweep /
// k_row_sweep (the reduced form of Algorithm 1, orthant cones), organised so that the gathers read
// shared memory instead of L2.
//
// The gathered vector (v for the column pass, x for the row pass) is cut into blocks of RB entries
// (64 KB of v, 96 KB of x in FP32). Each CTA owns a group of consecutive segments (columns or rows, balanced
// by nonzeros, at most a few ten thousand) and keeps one FP32 sum per segment in shared memory. It
// streams every block of the vector into shared memory in turn with bulk asynchronous copies
// (cp.async.bulk, two stages, an mbarrier each) and adds the products of its nonzeros whose
// gathered index falls in that block. The nonzeros of a group are therefore stored sorted by
// (block, segment, gathered index), one 8-byte entry each: the segment's index within the group in
// the low 16 bits, the gathered index within the block in the high 16 bits, and the FP32 value.
// Within one (group, block) the entries are cut into NW ranges, one per warp, at segment boundaries
// (precomputed), so that no two warps add into the same segment sum and every sum runs in a fixed
// order: blocks in turn, entries in order within a block. Each range is padded with zero entries of
// its last segment to a multiple of the entries one lane loads at once (LE: 6 for the column pass,
// about the 146 entries a warp takes per block in one 192-entry step; 4 for the row pass).
//
// Every CTA reads the whole vector once per pass (148 x 4 MB for a 10^6-row v), which L2 serves
// at about 28 TB/s to all SMs; the random gathers then cost shared-memory bank cycles instead of
// L2 sector requests. The nonzeros stream from HBM once, prefetched two blocks ahead into
// registers; the epilogue's inputs are prefetched into L2 (bulk prefetches) a few blocks before
// the group's last one, and its loads are batched so that several are in flight per thread.
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
#ifndef MFS_STG_NW
#define MFS_STG_NW 15
#endif
constexpr int RB_COL = MFS_STG_RB_COL;  // entries of v per block, column pass
constexpr int S_COL = MFS_STG_S_COL;    // stages
constexpr int RB_ROW = MFS_STG_RB_ROW;  // entries of x per block, row pass
constexpr int S_ROW = MFS_STG_S_ROW;
constexpr int ROW_HALVES = MFS_STG_ROW_HALVES;  // row pass: two CTAs per row group, each streaming
                                                // half of x (x is 2.5x longer than v)
constexpr int NW = MFS_STG_NW;  // consumer warps per CTA, plus one producer warp (15: 512 threads, 4 warps
                                // per SM sub-partition, up to 128 registers a thread)
constexpr int NTS = 32 * NW;
constexpr int MAXG = 24576;    // segments per group (their sums take 96 KB of shared memory)
#ifndef MFS_STG_LE_COL
#define MFS_STG_LE_COL 6
#define MFS_STG_PF_COL 1
#endif
#ifndef MFS_STG_LE_ROW
#define MFS_STG_LE_ROW 4
#define MFS_STG_PF_ROW 1
#endif
constexpr int LE_COL = MFS_STG_LE_COL;  // consecutive entries per lane and step (LE/4 32-byte loads)
constexpr int PF_COL = MFS_STG_PF_COL;  // steps of 32 * LE entries prefetched per warp and block
constexpr int LE_ROW = MFS_STG_LE_ROW;
constexpr int PF_ROW = MFS_STG_PF_ROW;
constexpr int EPI_U = 8;       // epilogue items per thread in flight
#ifndef MFS_STG_EPI_PF
#define MFS_STG_EPI_PF 4
#endif
#ifndef MFS_STG_PDL
#define MFS_STG_PDL 1
#endif
#ifndef MFS_STG_COMBINE_PF
#define MFS_STG_COMBINE_PF 1
#endif
constexpr int EPI_PF = MFS_STG_EPI_PF;  // blocks before a group's last one at which its epilogue's
                                        // inputs are prefetched into L2 (0: no prefetch)

// dynamic shared memory of one CTA: the vector stages, the group's sums, its split table, 2 S mbarriers
__host__ __device__ constexpr size_t smem_bytes(int rb, int stages, int maxg, int R) {
    return (size_t)stages * rb * 4 + (size_t)((maxg + 3) / 4 * 4) * 4 + (size_t)((R * (NW + 1) + 3) / 4 * 4) * 4 +
           (size_t)16 * stages;
}

struct StagedArgs {
    const int2* __restrict__ ent;   // entries, sorted by (group, block, segment, gathered index)
    const int* __restrict__ split;  // (G * R) x (NW + 1): warp ranges of each (group, block)
    const int* __restrict__ grp;    // G + 1: first segment of each group
    const int* __restrict__ wseg;   // G x (NW + 1): each warp's first segment within its group
    const float* __restrict__ vec;  // gathered vector, R * rb entries (tail padding unused)
    const float* __restrict__ rsq;  // row pass: sum of a_k^2 over each row
    int* err;                       // set to 1 if a wait for a block gave up
    int G, R, maxg_pad;
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
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
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

// A warp's range [s0, s1) (both multiples of LE) in steps of 32 * LE entries: lane l takes entries
// s0 + step*32*LE + l*LE .. +LE-1 with 32-byte loads (LE a multiple of 4) or 16-byte loads, words
// r[2*(step*LE + t)] (segment and gathered index) and r[2*(step*LE + t) + 1] (value bits) for t < LE;
// inactive lanes get zeros.
template <int PF, int LE>
__device__ __forceinline__ void load_lane(const int2* __restrict__ ent, int s0, int s1, int lane,
                                          int (&r)[2 * LE * PF], int nent) {
    static_assert(LE % 2 == 0, "entries per lane come in 16-byte pairs");
#pragma unroll
    for (int st = 0; st < PF; ++st) {
        int base = s0 + st * 32 * LE + lane * LE;
        if (base < s1 && !MFS_INB(base + LE - 1, nent, BS_STG_ENT)) base = s1;  // checked build: skip
        if (LE % 4 == 0) {  // 32-byte loads, bypassing L1 (each sector is used by one load)
#pragma unroll
            for (int h = 0; h < LE / 4; ++h) {
                const int q = 2 * (st * LE + 4 * h);
                if (base < s1) {
                    asm volatile("ld.global.nc.L1::no_allocate.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                 : "=r"(r[q + 0]), "=r"(r[q + 1]), "=r"(r[q + 2]), "=r"(r[q + 3]), "=r"(r[q + 4]),
                                   "=r"(r[q + 5]), "=r"(r[q + 6]), "=r"(r[q + 7])
                                 : "l"(ent + base + 4 * h));
                } else {
#pragma unroll
                    for (int w = 0; w < 8; ++w) r[q + w] = 0;
                }
            }
        } else {  // 16-byte loads through L1 (consecutive loads of a warp share sectors)
#pragma unroll
            for (int h = 0; h < LE / 2; ++h) {
                const int q = 2 * (st * LE + 2 * h);
                if (base < s1) {
                    asm volatile("ld.global.nc.v4.b32 {%0,%1,%2,%3}, [%4];"
                                 : "=r"(r[q + 0]), "=r"(r[q + 1]), "=r"(r[q + 2]), "=r"(r[q + 3])
                                 : "l"(ent + base + 2 * h));
                } else {
#pragma unroll
                    for (int w = 0; w < 4; ++w) r[q + w] = 0;
                }
            }
        }
    }
}

// One step of 32 * LE entries of a warp. Each lane forms the sums of the runs of equal segments
// among its LE entries (prefix sums that restart where the segment changes); a run that ends
// inside the lane's entries, other than its first, is added to the segment's sum at once. Runs that
// cross a lane boundary are joined: a lane whose first run continues the previous lane's last run
// adds that lane's partial sum to its own, and a lane whose last run continues into the next lane
// leaves it to that lane. A run through a whole lane (rare: more than LE entries of one segment)
// takes a segmented scan over the lanes' last runs instead. Either way every sum runs in the
// entries' order within the step, the same on every run; steps follow each other. A lane's runs
// belong to distinct segments, so their read-modify-writes are issued as all loads, then all stores.
template <int N, int LE, int RB>
__device__ __forceinline__ void lane_step(const int (&r)[N], int q0, bool active, const float* vb, float* acc,
                                          int lane, int nacc) {
    int k[LE];
    float s[LE];
#pragma unroll
    for (int t = 0; t < LE; ++t) {
        const uint32_t gi = (uint32_t)r[q0 + 2 * t] >> 16;
        const bool ok = active && MFS_INB(gi, RB, BS_STG_VEC) && MFS_INB(r[q0 + 2 * t] & 0xFFFF, nacc, BS_STG_ACC);
        k[t] = ok ? (r[q0 + 2 * t] & 0xFFFF) : -1;
        s[t] = ok ? __int_as_float(r[q0 + 2 * t + 1]) * vb[gi] : 0.f;
    }
#pragma unroll
    for (int t = 1; t < LE; ++t) s[t] += (k[t] == k[t - 1]) ? s[t - 1] : 0.f;
    bool mid[LE];
    bool seen = false;  // a run has ended before entry t
    float fs = s[LE - 1];
#pragma unroll
    for (int t = 0; t < LE - 1; ++t) {
        const bool end = k[t + 1] != k[t];
        mid[t] = active && end && seen;
        if (end && !seen) fs = s[t];
        seen = seen || end;
    }
    mid[LE - 1] = false;
    const bool single = !seen;
    const int fk = k[0], lk = k[LE - 1];
    const float ls = s[LE - 1];
    float old[LE];
#pragma unroll
    for (int t = 0; t < LE - 1; ++t)
        if (mid[t]) old[t] = acc[k[t]];
#pragma unroll
    for (int t = 0; t < LE - 1; ++t)
        if (mid[t]) acc[k[t]] = old[t] + s[t];
    const int pk = __shfl_up_sync(FULL, lk, 1);
    const float ps = __shfl_up_sync(FULL, ls, 1);
    const int nk = __shfl_down_sync(FULL, fk, 1);
    const bool cin = active && lane > 0 && pk == fk;
    const bool cout = active && lane < 31 && nk == lk;
    // firstv: the first run joined with the chain before the lane; lastv: the last run, joined with
    // that chain too when the lane holds a single run
    float firstv = fs + (cin ? ps : 0.f);
    float lastv = (single && cin) ? ls + ps : ls;
    if (__any_sync(FULL, single && cin && cout)) {
        // a run spans three or more lanes: join the lanes' last runs by a segmented scan
        float S = ls;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const float o = __shfl_up_sync(FULL, S, d);
            const int kk = __shfl_up_sync(FULL, lk, d);
            if (lane >= d && kk == lk) S += o;
        }
        const float sprev = __shfl_up_sync(FULL, S, 1);
        firstv = fs + (cin ? sprev : 0.f);
        lastv = S;
    }
    const bool wf = active && !single;  // first run, ending inside the lane
    const bool wl = active && !cout;    // last run, ending here
    const float of = wf ? acc[fk] : 0.f;
    const float ol = wl ? acc[lk] : 0.f;
    if (wf) acc[fk] = of + firstv;
    if (wl) acc[lk] = ol + lastv;
}

// All entries of a warp's range [s0, s1) of one block: PF prefetched steps, then any further ones.
template <int PF, int LE, int RB>
__device__ __forceinline__ void run_range(const int (&r)[2 * LE * PF], int s0, int s1, const int2* __restrict__ ent,
                                          const float* vb, float* acc, int lane, int nent, int nacc) {
#pragma unroll
    for (int st = 0; st < PF; ++st) {
        const int b0 = s0 + st * 32 * LE;
        if (b0 < s1) lane_step<2 * LE * PF, LE, RB>(r, 2 * LE * st, b0 + lane * LE < s1, vb, acc, lane, nacc);
        __syncwarp();
    }
    for (int b0 = s0 + PF * 32 * LE; b0 < s1; b0 += 32 * LE) {
        int t[2 * LE];
        load_lane<1, LE>(ent, b0, s1, lane, t, nent);
        lane_step<2 * LE, LE, RB>(t, 0, b0 + lane * LE < s1, vb, acc, lane, nacc);
        __syncwarp();
    }
}

// Block u of the CTA's sequence of staged blocks sits in stage u % S; full[k] completes when its
// copy has landed, empty[k] when every consumer warp has finished with it.
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Consumer side of block b (the CTA's block u): prefetch the warp's entries of block b + 2 into D,
// wait for the stage, add the entries held in C, and release the stage.
template <int RB, int PF, int LE, int S>
__device__ __forceinline__ void block_step(int b, int be, uint32_t u, int (&C)[2 * LE * PF], int (&D)[2 * LE * PF],
                                           const int* spl, const StagedArgs& g, const float* vb, float* acc,
                                           uint64_t* full, uint64_t* empty, bool& bad, int warp, int lane) {
    if (b + 2 < be) {
        const int* sp = spl + (b + 2) * (NW + 1) + warp;
        load_lane<PF, LE>(g.ent, sp[0], sp[1], lane, D, g.nent);
    }
    const uint32_t k = u % S;
    if (!wait_block(full + k, (u / S) & 1u, g.spin)) bad = true;
    const int* sp = spl + b * (NW + 1) + warp;
    run_range<PF, LE, RB>(C, sp[0], sp[1], g.ent, vb + k * RB, acc, lane, g.nent, g.maxg_pad);
    __syncwarp();
    if (lane == 0) mbar_arrive(empty + k);
}

// MODE 0: column pass (gathers v; epilogue x-, z-, delta-updates of orthant columns).
// MODE 1: row pass (gathers x; epilogue rho, lambda and v of each row).
// Warps 0..NW-1 consume; warp NW produces (its lane 0 issues the copies of the vector blocks).
// Warp w owns the segments wseg[w] .. wseg[w+1]-1 of its group in every block: it alone adds into
// their sums, and it runs their epilogue as soon as it has seen every block, while other warps
// may still be streaming.
template <int MODE, int RB, int PF, int LE, int S>
__global__ void __launch_bounds__(NTS + 32, 1) k_staged(const StagedArgs g, const SweepArgs<float> a) {
    constexpr int N = 2 * LE * PF;
    extern __shared__ __align__(128) unsigned char smem[];
    float* vb = reinterpret_cast<float*>(smem);
    float* acc = vb + S * RB;
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
        for (int t = threadIdx.x; t < R * (NW + 1); t += NTS + 32) spl[t] = gs[t];
        __syncthreads();  // split table in place; the previous group's sums are no longer read
        if (warp == NW) {
            dep_wait_prev();  // the vector was written by the previous pass
            if (lane == 0 && !g.no_loads) {
                for (int b = bb; b < be; ++b) {
                    const uint32_t u = u0 + (b - bb), k = u % S;
                    if (u >= S && !wait_block(empty + k, (u / S - 1) & 1u, g.spin)) bad = true;
                    issue_block(vb + k * RB, g.vec + (size_t)b * RB, RB * 4u, full + k);
                    if (EPI_PF > 0 && b == (be - EPI_PF > bb ? be - EPI_PF : bb)) {
                        // the group's epilogue reads these once every warp has seen all blocks
                        const size_t cnt = (size_t)(g.grp[grp + 1] - k0);
                        if (MODE == 0) {
                            prefetch_l2(a.x + k0, cnt * 4);
                            prefetch_l2(a.z + k0, cnt * 4);
                            prefetch_l2(a.del + k0, cnt * 4);
                            prefetch_l2(a.c + k0, cnt * 4);
                            prefetch_l2(a.col_ptr + k0, (cnt + 1) * 4);
                        } else if (H == 1) {
                            prefetch_l2(g.rsq + k0, cnt * 4);
                            prefetch_l2(a.b + k0, cnt * 4);
                            prefetch_l2(a.lam + k0, cnt * 4);
                        } else if (MFS_STG_COMBINE_PF) {  // for k_row_combine, split between the halves
                            if (h == 0) {
                                prefetch_l2(g.rsq + k0, cnt * 4);
                                prefetch_l2(a.b + k0, cnt * 4);
                            } else if (h == 1) {
                                prefetch_l2(a.lam + k0, cnt * 4);
                            }
                        }
                    }
                }
            }
        } else {
            const int ws = g.wseg[grp * (NW + 1) + warp], we = g.wseg[grp * (NW + 1) + warp + 1];
            for (int t = ws + lane; t < we; t += 32) acc[t] = 0.f;
            __syncwarp();
            int A[N], B[N], C[N];
            if (bb < be) load_lane<PF, LE>(g.ent, spl[bb * (NW + 1) + warp], spl[bb * (NW + 1) + warp + 1], lane, A, g.nent);
            if (bb + 1 < be)
                load_lane<PF, LE>(g.ent, spl[(bb + 1) * (NW + 1) + warp], spl[(bb + 1) * (NW + 1) + warp + 1], lane, B,
                                  g.nent);
            dep_wait_prev();  // the epilogue reads and writes the iterate
            for (int b = bb; b < be; b += 3) {
                const uint32_t u = u0 + (b - bb);
                block_step<RB, PF, LE, S>(b, be, u, A, C, spl, g, vb, acc, full, empty, bad, warp, lane);
                if (b + 1 < be)
                    block_step<RB, PF, LE, S>(b + 1, be, u + 1, B, A, spl, g, vb, acc, full, empty, bad, warp, lane);
                if (b + 2 < be)
                    block_step<RB, PF, LE, S>(b + 2, be, u + 2, C, B, spl, g, vb, acc, full, empty, bad, warp, lane);
            }
            __syncwarp();
            const float mu = a.mu;
            if (MODE == 0) {
                for (int t0 = ws + lane; t0 < we; t0 += 32 * EPI_U) {
                    float px[EPI_U], pz[EPI_U], pd[EPI_U], pc[EPI_U], dg[EPI_U];
#pragma unroll
                    for (int q = 0; q < EPI_U; ++q) {
                        const int t = t0 + q * 32;
                        if (t < we) {
                            const int j = k0 + t;
                            dg[q] = (float)(__ldg(a.col_ptr + j + 1) - __ldg(a.col_ptr + j));
                            px[q] = a.x[j];
                            pz[q] = a.z[j];
                            pd[q] = a.del[j];
                            pc[q] = __ldg(a.c + j);
                        }
                    }
#pragma unroll
                    for (int q = 0; q < EPI_U; ++q) {
                        const int t = t0 + q * 32;
                        if (t < we) {
                            const float xn = col_x_update(dg[q], px[q], acc[t], pz[q], pd[q], pc[q], mu);
                            orthant_update(a.x, a.z, a.del, k0 + t, xn, pd[q], mu);
                        }
                    }
                }
            } else if (H > 1) {  // partial row sums; k_row_combine adds the halves
                float* out = g.part + (size_t)h * g.nseg + k0;
                for (int t = ws + lane; t < we; t += 32) out[t] = acc[t];
            } else {
                for (int t0 = ws + lane; t0 < we; t0 += 32 * EPI_U) {
                    float pr[EPI_U], pb[EPI_U], pl[EPI_U];
#pragma unroll
                    for (int q = 0; q < EPI_U; ++q) {
                        const int t = t0 + q * 32;
                        if (t < we) {
                            const int i = k0 + t;
                            pr[q] = __ldg(g.rsq + i);
                            pb[q] = __ldg(a.b + i);
                            pl[q] = a.lam[i];
                        }
                    }
#pragma unroll
                    for (int q = 0; q < EPI_U; ++q) {
                        const int t = t0 + q * 32;
                        if (t < we) row_update<float, 0>(a, k0 + t, acc[t], pr[q], pb[q], pl[q]);
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

// Row pass with halves = 2: the two partial sums of each row, added in a fixed order, then rho,
// lambda and v (as the row pass's own epilogue).
__global__ void __launch_bounds__(256) k_row_combine(const StagedArgs g, const SweepArgs<float> a) {
    dep_launch_next();
    dep_wait_prev();
    const int m = g.nseg;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const float ax = g.part[i] + g.part[(size_t)m + i];
        row_update<float, 0>(a, i, ax, __ldg(g.rsq + i), __ldg(a.b + i), a.lam[i]);
    }
}

// the two instantiations the solver launches
#define MFS_STAGED_COL                                                                                  \
    ::mfs::staged::k_staged<0, ::mfs::staged::RB_COL, ::mfs::staged::PF_COL, ::mfs::staged::LE_COL, \
                            ::mfs::staged::S_COL>
#define MFS_STAGED_ROW                                                                                  \
    ::mfs::staged::k_staged<1, ::mfs::staged::RB_ROW, ::mfs::staged::PF_ROW, ::mfs::staged::LE_ROW, \
                            ::mfs::staged::S_ROW>

}  // namespace staged
}  // namespace mfs
