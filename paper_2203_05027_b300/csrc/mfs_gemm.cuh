// mfs_gemm.cuh -- dense BF16 GEMM on the 5th-generation tensor cores (tcgen05, sm_103a):
//   C[M x N] (+)= A[M x K] * B[N x K]^T      A, B row-major BF16 (both K-major), FP32 accumulate.
//
// One CTA computes one 128 x 128 tile of C (or a K-slice of it, for split-K). Eight warps:
//   warp 0, one lane: TMA producer, 2-D tiled loads of 128 x 64 BF16 boxes of A and B into a
//                     STAGES-deep ring of shared-memory stages (128-byte swizzle);
//   warp 1, one lane: issues tcgen05.mma (M = 128, N = 128, K = 16 per instruction) from shared
//                     memory descriptors into a 128 x 128 FP32 accumulator in tensor memory;
//   all eight warps:  epilogue, tcgen05.ld of their 32 accumulator lanes (rows) and 64 columns, a transpose through
//                     shared memory, bias, ReLU, conversion and row-contiguous stores.
// Barriers: full[s] (TMA transaction bytes), empty[s] (tcgen05.commit after the MMAs that read
// stage s), acc (commit after the last MMA). Every wait is bounded: a wait that runs out sets the
// error word and the kernel skips to the end, where tensor memory is freed.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cstdint>

#include "mfs_device.cuh"

namespace mfs {
namespace gemm {

constexpr int BM = 128;
constexpr int BN = 128;
constexpr int BK = 64;       // one 128-byte swizzle row of BF16
constexpr int UK = 16;       // K of one tcgen05.mma kind::f16
constexpr int STAGES = 3;       // 3 stages (97 KB) let two CTAs share an SM: one's epilogue overlaps the other's loads
constexpr int NTHREADS = 256;  // eight warps: warp w reads TMEM lanes 32 (w % 4) .. +31, columns of half w / 4
constexpr int TILE_A = BM * BK * 2;  // bytes
constexpr int TILE_B = BN * BK * 2;
constexpr int STAGE_BYTES = TILE_A + TILE_B;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /* alignment */ + 256 /* barriers */;
constexpr uint32_t SPIN = 1u << 24;
constexpr int ERR_TIMEOUT = 2;

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

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

// Bounded wait by the calling thread (at most `limit` polls); false if the phase never completed.
__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t parity, uint32_t limit = SPIN) {
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Shared-memory matrix descriptor (tcgen05): K-major operand tile in the canonical 128-byte
// swizzled layout (rows of 128 bytes, 8-row groups 1024 bytes apart).
__device__ __forceinline__ uint64_t smem_desc(const void* p) {
    const uint64_t addr = smem_addr(p);
    uint64_t d = 0;
    d |= (addr >> 4) & 0x3FFFull;         // start address
    d |= (uint64_t)1 << 16;               // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;     // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;               // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;               // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 32 consecutive FP32 accumulator columns of this thread's lane (row).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

struct GemmArgs {
    int M, N, K;
    int kblocks_per_split;  // K blocks handled by one CTA (gridDim.z slices)
    const float* bias;      // N, or nullptr (applied only when splits == 1)
    int relu;               // apply ReLU (only when splits == 1)
    int out_fp32;           // C element type: FP32 if set, else BF16
    void* C;                // row-major M x N; with splits > 1: FP32 partials [split][M][N]
    int ldc;
    int* err;
    uint32_t spin;  // poll limit of every wait (SPIN in normal use)
    int m_fast;     // blockIdx.x runs over row tiles (B tiles shared by neighbouring CTAs), else column tiles
    int no_loads;   // diagnostic: issue no loads, so the first wait of the MMA issuer runs out
    // EPI_LOSS: y = acc + bias; r = y - (T[row][col] - mean[col]) / stdv[col] for col < dout (else 0);
    // dY[row][col] (ld ldc, in C) and dYt[col][row] (ld ldt) receive bf16(scale r); per-CTA sums of r^2
    // go to part[] (C never holds y).
    const float* T;
    int ldT, dout;
    const float *mean, *stdv;
    float scale;
    __nv_bfloat16* dYt;
    int ldt;
    double* part;
    // EPI_ADAM: g = acc is the gradient of W [row][col] (ld ldc); Adam updates W and its moments and
    // refreshes the BF16 copies Wh [row][col] (ld ldc) and Wt [col][row] (ld ldt).
    float *W, *mom, *vel;
    __nv_bfloat16 *Wh, *Wt;
    float lr, b1, b2, eps, c1, c2;
    float* gkeep;  // EPI_ADAM: nullable; receives the gradient g [row][col] (ld ldc) as well
};

enum { EPI_STORE = 0, EPI_LOSS = 1, EPI_ADAM = 2 };

// Hint: bring the 16-byte-aligned part of [p, p + bytes) into L2 (a bulk prefetch; nothing outside
// the range is touched, nothing waits for it).
__device__ __forceinline__ void gemm_prefetch_l2(const void* p, size_t bytes) {
    const uintptr_t s = ((uintptr_t)p + 15) & ~(uintptr_t)15, e = ((uintptr_t)p + bytes) & ~(uintptr_t)15;
    if (e > s) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(s), "r"((uint32_t)(e - s)) : "memory");
}

// The epilogue of one 32-column block of the accumulator tile (columns n0 + c0 .. + 31, rows rbase ..
// rbase + 31), by one warp whose staging block stg (32 x 33 floats) holds it with lane = row:
// bias, ReLU and the store (EPI_STORE; FP32 partials with part), or the loss or the Adam update
// (lane = column, rows in turn) followed by the transposed BF16 store (lane = row).
template <int EPI>
__device__ __forceinline__ void epi_block(const GemmArgs& g, float* stg, int lane, int rbase, int n0, int c0, bool part,
                                          double& lsum) {
    const int col = n0 + c0 + lane;
    const int rows = min(32, g.M - rbase);
    if (EPI == EPI_STORE) {
        if (col < g.N) {
            const float bv = (!part && g.bias) ? g.bias[col] : 0.f;
            for (int r = 0; r < rows; ++r) {
                const size_t row = (size_t)(rbase + r);
                float w = stg[r * 33 + lane];
                if (part) {
                    reinterpret_cast<float*>(g.C)[((size_t)blockIdx.z * g.M + row) * g.ldc + col] = w;
                } else {
                    w += bv;
                    if (g.relu) w = w > 0.f ? w : 0.f;
                    if (g.out_fp32)
                        reinterpret_cast<float*>(g.C)[row * g.ldc + col] = w;
                    else
                        reinterpret_cast<__nv_bfloat16*>(g.C)[row * g.ldc + col] = __float2bfloat16_rn(w);
                }
            }
        }
    } else {
        // EPI_LOSS / EPI_ADAM: lane = column, rows in turn; the BF16 result goes back to the
        // staging block for the transposed store below
        if (col < g.N) {
            // eight rows at a time: their loads are issued together, then used
            if (EPI == EPI_LOSS) {
                const bool real = col < g.dout;
                const float bv = g.bias ? g.bias[col] : 0.f;
                const float mc = real ? g.mean[col] : 0.f, sc = real ? g.stdv[col] : 1.f;
                // the lane's squares summed in FP32 over its (at most 32) rows, then added into the
                // FP64 sum once: FP64 runs at 1/64 of the FP32 rate on this GPU
                float fs = 0.f;
                for (int r0 = 0; r0 < rows; r0 += 8) {
                    float tv[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        tv[u] = (real && r0 + u < rows) ? g.T[(size_t)(rbase + r0 + u) * g.ldT + col] : 0.f;
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int r = r0 + u;
                        if (r < rows) {
                            const float y = stg[r * 33 + lane] + bv;
                            float res = 0.f;
                            if (real) res = y - (tv[u] - mc) / sc;
                            fs = fmaf(res, res, fs);
                            const __nv_bfloat16 d = __float2bfloat16_rn(g.scale * res);
                            reinterpret_cast<__nv_bfloat16*>(g.C)[(size_t)(rbase + r) * g.ldc + col] = d;
                            stg[r * 33 + lane] = __bfloat162float(d);
                        }
                    }
                }
                lsum += (double)fs;
            } else {
                // the bias corrections' reciprocals, once (a multiplication instead of a division
                // per element: the same steps, FP32 rounding of their own)
                const float rc1 = 1.f / g.c1, rc2 = 1.f / g.c2;
                for (int r0 = 0; r0 < rows; r0 += 8) {
                    float wv[8], mv[8], vv[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        if (r0 + u < rows) {
                            const size_t idx = (size_t)(rbase + r0 + u) * g.ldc + col;
                            wv[u] = g.W[idx];
                            mv[u] = g.mom[idx];
                            vv[u] = g.vel[idx];
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int r = r0 + u;
                        if (r < rows) {
                            const size_t idx = (size_t)(rbase + r) * g.ldc + col;
                            const float gt = stg[r * 33 + lane];
                            if (g.gkeep) g.gkeep[idx] = gt;
                            const float mt = g.b1 * mv[u] + (1.f - g.b1) * gt;
                            const float vt = g.b2 * vv[u] + (1.f - g.b2) * gt * gt;
                            g.mom[idx] = mt;
                            g.vel[idx] = vt;
                            const float wn = wv[u] - g.lr * (mt * rc1) / (sqrtf(vt * rc2) + g.eps);
                            g.W[idx] = wn;
                            const __nv_bfloat16 h = __float2bfloat16_rn(wn);
                            g.Wh[idx] = h;
                            stg[r * 33 + lane] = __bfloat162float(h);
                        }
                    }
                }
            }
        }
        __syncwarp();
        // transposed store: lane = row, columns in turn
        const int row = rbase + lane;
        __nv_bfloat16* dst = EPI == EPI_LOSS ? g.dYt : g.Wt;
        if (row < g.M)
            for (int i = 0; i < 32; ++i) {
                const int cc = n0 + c0 + i;
                if (cc < g.N) dst[(size_t)cc * g.ldt + row] = __float2bfloat16_rn(stg[lane * 33 + i]);
            }
    }
}

template <int EPI>
__global__ void __launch_bounds__(NTHREADS, 2)
    k_gemm_bf16(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, const GemmArgs g) {
    extern __shared__ __align__(1024) unsigned char gsm_raw[];
    unsigned char* gsm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(gsm_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(gsm + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* accb = empty + STAGES;
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(accb + 1);
    int* s_fail = reinterpret_cast<int*>(s_tmem + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = (g.m_fast ? blockIdx.y : blockIdx.x) * BN, m0 = (g.m_fast ? blockIdx.x : blockIdx.y) * BM;
    const int kb_total = (g.K + BK - 1) / BK;
    const int kb0 = blockIdx.z * g.kblocks_per_split;
    const int kb1 = min(kb_total, kb0 + g.kblocks_per_split);
    const int nkb = max(0, kb1 - kb0);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accb, 1);
        *s_fail = 0;
        fence_mbar_init();
    }
    if (warp == 0) {  // tensor memory for the 128 x 128 FP32 accumulator (128 columns)
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(s_tmem)),
                     "r"(BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;
    // The fused epilogues read a tile of FP32 data besides the accumulator (the targets; W and its
    // moments): the warps that wait for the accumulator prefetch those rows into L2 now, so that the
    // epilogue's loads, issued after the short main loop (K <= 512), find them there.
    if (EPI != EPI_STORE && gridDim.z == 1 && warp >= 2) {
        const int t = (warp - 2) * 32 + lane, row = m0 + t;
        if (t < BM && row < g.M) {
            if (EPI == EPI_LOSS) {
                const int c1 = min(n0 + BN, g.dout);
                if (c1 > n0) gemm_prefetch_l2(g.T + (size_t)row * g.ldT + n0, (size_t)(c1 - n0) * sizeof(float));
            } else {
                const int c1 = min(n0 + BN, g.N);
                if (c1 > n0) {
                    const size_t off = (size_t)row * g.ldc + n0, bytes = (size_t)(c1 - n0) * sizeof(float);
                    gemm_prefetch_l2(g.W + off, bytes);
                    gemm_prefetch_l2(g.mom + off, bytes);
                    gemm_prefetch_l2(g.vel + off, bytes);
                }
            }
        }
    }

    int issued = 0;                // loads issued by the producer lane
    if (warp == 0 && lane == 0) {  // producer
        for (int i = 0; i < nkb && !g.no_loads; ++i) {
            const int s = i % STAGES;
            if (!wait_phase(&empty[s], ((i / STAGES) & 1) ^ 1, g.spin)) {
                atomicExch(s_fail, 1);
                break;
            }
            unsigned char* st = gsm + s * STAGE_BYTES;
            mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
            tma_load_2d(st, &mapA, (kb0 + i) * BK, m0, &full[s]);
            tma_load_2d(st + TILE_A, &mapB, (kb0 + i) * BK, n0, &full[s]);
            issued = i + 1;
        }
    } else if (warp == 1 && lane == 0) {  // MMA issuer
        const uint32_t idesc = idesc_bf16(BM, BN);
        for (int i = 0; i < nkb; ++i) {
            const int s = i % STAGES;
            if (!wait_phase(&full[s], (i / STAGES) & 1, g.spin)) {
                atomicExch(s_fail, 1);
                break;
            }
            tc_fence_after();
            unsigned char* st = gsm + s * STAGE_BYTES;
#pragma unroll
            for (int kk = 0; kk < BK / UK; ++kk) {
                const uint64_t ad = smem_desc(st + kk * UK * 2);
                const uint64_t bd = smem_desc(st + TILE_A + kk * UK * 2);
                mma_bf16(tmem, ad, bd, idesc, (i > 0 || kk > 0) ? 1u : 0u);
            }
            mma_commit(&empty[s]);  // stage s is free once these MMAs have read it
        }
        mma_commit(accb);  // the accumulator is complete once all issued MMAs are
    }
    __syncwarp();
    // epilogue: every thread owns one row of the tile (TMEM lane = row)
    const bool ok = wait_phase(accb, 0, g.spin);
    if (!ok) atomicExch(s_fail, 1);
    tc_fence_after();
    // Each 32 x 32 block goes through shared memory (the idle stage buffers; padded rows, no bank
    // conflicts) so that each store instruction writes 32 consecutive columns of one row.
    float* stg = reinterpret_cast<float*>(gsm) + warp * (32 * 33);
    const int quad = warp & 3, half = warp >> 2;  // TMEM lane quadrant (rows) and column half
    const int rbase = m0 + quad * 32;
    const bool part = gridDim.z > 1;
    double lsum = 0.0;  // EPI_LOSS: this thread's share of the squared residuals
    if (ok && nkb > 0 && !*s_fail) {
        for (int c0 = half * (BN / 2); c0 < (half + 1) * (BN / 2); c0 += 32) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
            for (int i = 0; i < 32; ++i) stg[lane * 33 + i] = v[i];
            __syncwarp();
            epi_block<EPI>(g, stg, lane, rbase, n0, c0, part, lsum);
            __syncwarp();
        }
    }
    if (EPI == EPI_LOSS) {  // fixed-order sum of the CTA's squared residuals
        double* red = reinterpret_cast<double*>(gsm + (NTHREADS / 32) * (32 * 33) * sizeof(float));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, o);
        if (lane == 0) red[warp] = lsum;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < NTHREADS / 32; ++w) t += red[w];
            g.part[blockIdx.y * gridDim.x + blockIdx.x] = t;
        }
    }
    tc_fence_before();
    __syncthreads();  // every role is done: s_fail is final
    if (*s_fail) {
        // Before the CTA's shared and tensor memory go away: the bulk copies still in flight (only
        // the last STAGES issued can be, the earlier ones were consumed) and the issued MMAs.
        if (warp == 0 && lane == 0)
            for (int i = max(0, issued - STAGES); i < issued; ++i) wait_phase(&full[i % STAGES], (i / STAGES) & 1);
        if (threadIdx.x == 32) wait_phase(accb, 0);
        if (threadIdx.x == 0) atomicCAS(g.err, 0, ERR_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
}


// ---------------------------------------------------------------------------------------------
// Persistent form for the fused epilogues (EPI_LOSS, EPI_ADAM; no split-K). One CTA per SM loops
// over the 128 x 128 tiles in the one-tile kernel's order (tile t = blockIdx.y * gridDim.x +
// blockIdx.x of its grid), so that a tile's epilogue overlaps the loads and MMAs of the next:
//   warp 0, one lane: TMA producer, a PSTAGES-deep ring of stages that runs on across tiles;
//   warp 1, one lane: MMA issuer, tile j into accumulator j % 2 (two 128-column accumulators in
//                     tensor memory), after the epilogue has read that accumulator's tile j - 2;
//   warps 2 .. 2 + PEW - 1: the epilogue, each warp 32 rows (its TMEM lane quadrant) and
//                     128 / (PEW / 4) columns of the tile, through its own staging block.
// Barriers: full/empty per stage (as in k_gemm_bf16), tfull[a] (commit after the tile's last MMA),
// tempty[a] (one arrival per epilogue warp once its tcgen05.ld of the tile have completed). The
// loss's per-tile sum of squares is added in the one-tile kernel's warp order. Every wait is
// bounded; one that runs out sets the error word and every role leaves its loop; the CTA then
// waits for its MMAs and copies in flight before it frees tensor memory.
#ifndef MFS_GEMM_PEW
#define MFS_GEMM_PEW 16
#endif
constexpr int PSTAGES = 4;
constexpr int PEW = MFS_GEMM_PEW;             // epilogue warps: 8 or 16
constexpr int PCOLS = BN / (PEW / 4);         // accumulator columns per epilogue warp
constexpr int PTHREADS = 32 * (2 + PEW);
constexpr int PSTG_BYTES = PEW * 32 * 33 * 4;  // the epilogue warps' staging blocks
constexpr int PSMEM_BYTES = PSTAGES * STAGE_BYTES + PSTG_BYTES + 1024 /* alignment */ + 512 /* barriers */;
static_assert(PEW == 8 || PEW == 16, "epilogue warps");

__device__ __forceinline__ void mbar_arrive1(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// L2 prefetch of the epilogue's FP32 inputs for rows [r0, r0 + 32) x columns [c0, c0 + PCOLS) of a tile
template <int EPI>
__device__ __forceinline__ void prefetch_epi_rows(const GemmArgs& g, int row, int c0) {
    if (row >= g.M) return;
    if (EPI == EPI_LOSS) {
        const int c1 = min(c0 + PCOLS, g.dout);
        if (c1 > c0) gemm_prefetch_l2(g.T + (size_t)row * g.ldT + c0, (size_t)(c1 - c0) * sizeof(float));
    } else {
        const int c1 = min(c0 + PCOLS, g.N);
        if (c1 > c0) {
            const size_t off = (size_t)row * g.ldc + c0, bytes = (size_t)(c1 - c0) * sizeof(float);
            gemm_prefetch_l2(g.W + off, bytes);
            gemm_prefetch_l2(g.mom + off, bytes);
            gemm_prefetch_l2(g.vel + off, bytes);
        }
    }
}

template <int EPI>
__global__ void __launch_bounds__(PTHREADS, 1)
    k_gemm_bf16_pers(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                     const GemmArgs g) {
    extern __shared__ __align__(1024) unsigned char gsm_raw[];
    unsigned char* gsm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(gsm_raw) + 1023) & ~uintptr_t(1023));
    float* stg_all = reinterpret_cast<float*>(gsm + PSTAGES * STAGE_BYTES);
    uint64_t* full = reinterpret_cast<uint64_t*>(gsm + PSTAGES * STAGE_BYTES + PSTG_BYTES);
    uint64_t* empty = full + PSTAGES;
    uint64_t* tfull = empty + PSTAGES;
    uint64_t* tempty = tfull + 2;
    uint64_t* dbar = tempty + 2;
    uint64_t* rfull = dbar + 1;  // EPI_LOSS: red[b] holds every epilogue warp's sum (b = tile % 2)
    uint64_t* rfree = rfull + 2;  //           red[b] has been added up and may take the next tile's
    double* red = reinterpret_cast<double*>(rfree + 2);  // 2 x PEW
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(red + 2 * PEW);
    int* s_fail = reinterpret_cast<int*>(s_tmem + 1);
    volatile int* vfail = s_fail;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mt = (g.M + BM - 1) / BM, nt = (g.N + BN - 1) / BN, T = mt * nt;
    const int nkb = (g.K + BK - 1) / BK;
    auto tile_of = [&](int t, int& m0, int& n0) {
        if (g.m_fast) {
            m0 = (t % mt) * BM;
            n0 = (t / mt) * BN;
        } else {
            m0 = (t / nt) * BM;
            n0 = (t % nt) * BN;
        }
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < PSTAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], PEW);
        }
        mbar_init(dbar, 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(&rfull[b], PEW);
            mbar_init(&rfree[b], 1);
        }
        *s_fail = 0;
        fence_mbar_init();
    }
    if (warp == 0) {  // two 128 x 128 FP32 accumulators (256 columns)
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(s_tmem)),
                     "r"(2 * BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;

    int issued = 0;   // producer: loads issued
    bool mmas = false;  // MMA issuer: any MMA issued
    if (warp == 0) {
        if (lane == 0 && !g.no_loads) {
            int it = 0;
            bool stop = false;
            for (int t = blockIdx.x; t < T && !stop; t += gridDim.x) {
                int m0, n0;
                tile_of(t, m0, n0);
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = it % PSTAGES;
                    if (*vfail || !wait_phase(&empty[s], ((it / PSTAGES) & 1) ^ 1, g.spin)) {
                        atomicExch(s_fail, 1);
                        stop = true;
                        break;
                    }
                    unsigned char* st = gsm + s * STAGE_BYTES;
                    mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
                    tma_load_2d(st, &mapA, kb * BK, m0, &full[s]);
                    tma_load_2d(st + TILE_A, &mapB, kb * BK, n0, &full[s]);
                    issued = it + 1;
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(BM, BN);
            int it = 0, j = 0;
            for (int t = blockIdx.x; t < T; t += gridDim.x, ++j) {
                const int a = j & 1;
                if (*vfail || !wait_phase(&tempty[a], ((j >> 1) & 1) ^ 1, g.spin)) {
                    atomicExch(s_fail, 1);
                    break;
                }
                tc_fence_after();
                const uint32_t acc = tmem + (uint32_t)(a * BN);
                bool stop = false;
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = it % PSTAGES;
                    if (!wait_phase(&full[s], (it / PSTAGES) & 1, g.spin)) {
                        atomicExch(s_fail, 1);
                        stop = true;
                        break;
                    }
                    tc_fence_after();
                    unsigned char* st = gsm + s * STAGE_BYTES;
#pragma unroll
                    for (int kk = 0; kk < BK / UK; ++kk) {
                        const uint64_t ad = smem_desc(st + kk * UK * 2);
                        const uint64_t bd = smem_desc(st + TILE_A + kk * UK * 2);
                        mma_bf16(acc, ad, bd, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
                    }
                    mmas = true;
                    mma_commit(&empty[s]);  // the stage is free once these MMAs have read it
                }
                if (stop) break;
                mma_commit(&tfull[a]);  // the tile's accumulator is complete once its MMAs are
            }
        }
        __syncwarp();
    } else {
        const int ew = warp - 2;
        const int quad = warp & 3, part4 = ew >> 2;  // TMEM lane quadrant (rows) and column part
        const int cbase = part4 * PCOLS;
        float* stg = stg_all + ew * (32 * 33);
        int j = 0;
        {
            int m0, n0;
            if (blockIdx.x < T) {
                tile_of(blockIdx.x, m0, n0);
                prefetch_epi_rows<EPI>(g, m0 + quad * 32 + lane, n0 + cbase);
            }
        }
        for (int t = blockIdx.x; t < T; t += gridDim.x, ++j) {
            int m0, n0;
            tile_of(t, m0, n0);
            const int a = j & 1;
            // a warp-uniform decision: the tensor-memory loads below need every lane
            const int okw = __all_sync(0xffffffffu, !*vfail && wait_phase(&tfull[a], (j >> 1) & 1, g.spin));
            if (!okw) {
                if (lane == 0) atomicExch(s_fail, 1);
                break;
            }
            tc_fence_after();
            if (t + (int)gridDim.x < T) {  // the next tile's epilogue inputs into L2
                int m1, n1;
                tile_of(t + gridDim.x, m1, n1);
                prefetch_epi_rows<EPI>(g, m1 + quad * 32 + lane, n1 + cbase);
            }
            float v[PCOLS];
            const uint32_t ta = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(a * BN + cbase);
#pragma unroll
            for (int c = 0; c < PCOLS; c += 32) {
                float w[32];
                tmem_ld32(ta + (uint32_t)c, w);
#pragma unroll
                for (int i = 0; i < 32; ++i) v[c + i] = w[i];
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive1(&tempty[a]);  // the accumulator may take tile j + 2
            const int rbase = m0 + quad * 32;
            double lsum = 0.0;
#pragma unroll
            for (int c = 0; c < PCOLS; c += 32) {
#pragma unroll
                for (int i = 0; i < 32; ++i) stg[lane * 33 + i] = v[c + i];
                __syncwarp();
                epi_block<EPI>(g, stg, lane, rbase, n0, cbase + c, false, lsum);
                __syncwarp();
            }
            if (EPI == EPI_LOSS) {
                // the tile's sum of squares: every warp's share into red[b] (once the tile two back
                // has been added up), then warp 2 adds them in the one-tile kernel's order (column
                // half, lane quadrant) and writes part[t]; bounded waits on mbarriers only
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, o);
                const int b = j & 1;
                if (lane == 0) {
                    if (!wait_phase(&rfree[b], ((j >> 1) & 1) ^ 1, g.spin)) atomicExch(s_fail, 1);
                    red[b * PEW + quad * (PEW / 4) + part4] = lsum;
                    mbar_arrive1(&rfull[b]);
                    if (ew == 0) {
                        if (wait_phase(&rfull[b], (j >> 1) & 1, g.spin)) {
                            double tsum = 0.0;
                            for (int h = 0; h < 2; ++h)
                                for (int q = 0; q < 4; ++q)
                                    for (int pp = h * (PEW / 8); pp < (h + 1) * (PEW / 8); ++pp)
                                        tsum += red[b * PEW + q * (PEW / 4) + pp];
                            g.part[t] = tsum;
                        } else {
                            atomicExch(s_fail, 1);
                        }
                        mbar_arrive1(&rfree[b]);
                    }
                }
                __syncwarp();
            }
        }
    }
    // the MMAs issued (all complete once this commit arrives) before tensor memory is freed
    if (warp == 1 && lane == 0 && mmas) {
        mma_commit(dbar);
        wait_phase(dbar, 0);
    }
    tc_fence_before();
    __syncthreads();
    if (*s_fail) {
        // copies still in flight (only the last PSTAGES issued can be)
        if (warp == 0 && lane == 0)
            for (int i = max(0, issued - PSTAGES); i < issued; ++i) wait_phase(&full[i % PSTAGES], (i / PSTAGES) & 1);
        if (threadIdx.x == 0) atomicCAS(g.err, 0, ERR_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * BN) : "memory");
}

}  // namespace gemm
}  // namespace mfs
