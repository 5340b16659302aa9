// mfs_mlp.cu -- the learned warm start: a 3-layer BF16 MLP (theta -> width -> width -> n+m) whose
// forward and backward GEMMs run on the tcgen05 kernel of mfs_gemm.cuh, with FP32 master weights
// and Adam. The network is trained on solutions that the solver itself produced and maps a
// problem's parameters to an initial (x, lambda) for mfs_warm_start.
//
// Layout: weights W_l row-major [out][in] (FP32 master, BF16 copy, BF16 transposed copy for the
// backward GEMMs); activations row-major [batch][features] in BF16; outputs and gradients of
// weights in FP32. Every GEMM is C = A * B^T with both operands K-major, so the backward pass
// transposes the operands it needs (tiled shared-memory transposes) instead of using MN-major
// tensor-core layouts.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/mfs.h"
#include "mfs_trace.h"
#include "mfs_alloc.h"
#include "mfs_gemm.cuh"

using bf16 = __nv_bfloat16;

namespace {

using namespace mfs::gemm;

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
    static EncodeFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
    }
    return fn;
}

// Tensor map of a row-major BF16 matrix [rows][cols] read in boxes of 128 rows x 64 columns with
// the 128-byte swizzle (out-of-bounds elements read as zero).
bool make_map(CUtensorMap* map, const void* base, int rows, int cols) {
    EncodeFn enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, 128};
    cuuint32_t es[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Sum of split-K partials [splits][M][N] (+ bias, ReLU) into C (FP32 or BF16).
__global__ void k_splitk_reduce(const float* __restrict__ part, int splits, int M, int N, const float* __restrict__ bias,
                                int relu, int out_fp32, void* C) {
    const long long total = (long long)M * N;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        float v = 0.f;
        for (int s = 0; s < splits; ++s) v += part[(size_t)s * total + t];
        if (bias) v += bias[t % N];
        if (relu) v = v > 0.f ? v : 0.f;
        if (out_fp32)
            reinterpret_cast<float*>(C)[t] = v;
        else
            reinterpret_cast<bf16*>(C)[t] = __float2bfloat16_rn(v);
    }
}

// C (row-major M x N) = A (M x K) * B (N x K)^T, BF16 in, FP32 accumulate on the tensor cores.
template <int EPI>
bool gemm_attr() {
    static bool done = false;
    if (!done)
        done = cudaFuncSetAttribute(k_gemm_bf16<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES) ==
               cudaSuccess;
    return done;
}

// Fused epilogues in the persistent GEMM (one CTA per SM, two accumulators in tensor memory, each
// tile's epilogue overlapping the next tile's loads and MMAs): 0 none, 1 the loss, 2 the loss and Adam.
#ifndef MFS_GEMM_PERSISTENT
#define MFS_GEMM_PERSISTENT 1
#endif
template <int EPI>
bool gemm_pers_attr() {
    static bool done = false;
    if (!done)
        done = cudaFuncSetAttribute(k_gemm_bf16_pers<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    PSMEM_BYTES) == cudaSuccess;
    return done;
}

int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
            n = 148;
    }
    return n;
}

// epi != EPI_STORE: the fused epilogue's fields are taken from *fused (splits must be 1).
mfs_status gemm(int M, int N, int K, const bf16* A, const bf16* B, const float* bias, int relu, int out_fp32, void* C,
                int splits, float* work, int* err, cudaStream_t st, std::string* why, uint32_t spin = SPIN,
                int no_loads = 0, int epi = EPI_STORE, const GemmArgs* fused = nullptr) {
    if (M <= 0 || N <= 0 || K <= 0) return MFS_OK;
    if (K % 8) {
        if (why) *why = "gemm: K must be a multiple of 8 (16-byte rows)";
        return MFS_ERR_INVALID;
    }
    if (!gemm_attr<EPI_STORE>() || !gemm_attr<EPI_LOSS>() || !gemm_attr<EPI_ADAM>()) {
        if (why) *why = "gemm: shared memory attribute";
        return MFS_ERR_CUDA;
    }
    if (epi != EPI_STORE && (!fused || splits != 1)) {
        if (why) *why = "gemm: a fused epilogue needs its arguments and no split-K";
        return MFS_ERR_INVALID;
    }
    CUtensorMap ma, mb;
    if (!make_map(&ma, A, M, K) || !make_map(&mb, B, N, K)) {
        if (why) *why = "gemm: cuTensorMapEncodeTiled failed";
        return MFS_ERR_CUDA;
    }
    const int kbt = (K + BK - 1) / BK;
    splits = std::max(1, std::min(splits, kbt));
    const int kbps = (kbt + splits - 1) / splits;
    splits = (kbt + kbps - 1) / kbps;
    if (splits > 1 && !work) {
        if (why) *why = "gemm: split-K needs a workspace";
        return MFS_ERR_INVALID;
    }
    GemmArgs g = fused ? *fused : GemmArgs{};
    g.M = M;
    g.N = N;
    g.K = K;
    g.kblocks_per_split = kbps;
    g.bias = splits > 1 ? nullptr : bias;
    g.relu = splits > 1 ? 0 : relu;
    g.out_fp32 = out_fp32;
    g.C = splits > 1 ? static_cast<void*>(work) : C;
    g.ldc = N;
    g.err = err;
    g.spin = spin;
    g.no_loads = no_loads;
    // neighbouring CTAs share the tiles of the larger operand, so it is read from DRAM about once
    g.m_fast = (long long)N > (long long)M ? 1 : 0;
    const int mt = (M + BM - 1) / BM, nt = (N + BN - 1) / BN;
    dim3 grid(g.m_fast ? mt : nt, g.m_fast ? nt : mt, splits);
    if ((MFS_GEMM_PERSISTENT >= 1 && epi == EPI_LOSS) || (MFS_GEMM_PERSISTENT >= 2 && epi == EPI_ADAM)) {
        if (!gemm_pers_attr<EPI_LOSS>() || !gemm_pers_attr<EPI_ADAM>()) {
            if (why) *why = "gemm: shared memory attribute";
            return MFS_ERR_CUDA;
        }
        const int pgrid = std::max(1, std::min(mt * nt, sm_count()));
        if (epi == EPI_LOSS)
            k_gemm_bf16_pers<EPI_LOSS><<<pgrid, PTHREADS, PSMEM_BYTES, st>>>(ma, mb, g);
        else
            k_gemm_bf16_pers<EPI_ADAM><<<pgrid, PTHREADS, PSMEM_BYTES, st>>>(ma, mb, g);
    } else if (epi == EPI_LOSS)
        k_gemm_bf16<EPI_LOSS><<<grid, NTHREADS, SMEM_BYTES, st>>>(ma, mb, g);
    else if (epi == EPI_ADAM)
        k_gemm_bf16<EPI_ADAM><<<grid, NTHREADS, SMEM_BYTES, st>>>(ma, mb, g);
    else
        k_gemm_bf16<EPI_STORE><<<grid, NTHREADS, SMEM_BYTES, st>>>(ma, mb, g);
    if (splits > 1) {
        const long long total = (long long)M * N;
        const int blocks = (int)std::min<long long>((total + 255) / 256, 148 * 8);
        k_splitk_reduce<<<blocks, 256, 0, st>>>(work, splits, M, N, bias, relu, out_fp32, C);
    }
    if (cudaGetLastError() != cudaSuccess) {
        if (why) *why = "gemm: launch failed";
        return MFS_ERR_CUDA;
    }
    return MFS_OK;
}

// Tiled transpose: out[c][r] = in[r][c] for a row-major BF16 matrix [rows][cols]. A 64 x 64 tile
// moves as pairs of BF16 (4-byte accesses, 128 bytes per warp row) through shared memory.
__global__ void k_transpose(const bf16* __restrict__ in, bf16* __restrict__ out, int rows, int cols) {
    __shared__ bf16 tile[64][66];
    const int tx = threadIdx.x;  // 0..31: a pair of columns (load) or of rows (store)
    const int c0 = blockIdx.x * 64, r0 = blockIdx.y * 64;
    const bool pair_in = (cols % 2 == 0), pair_out = (rows % 2 == 0);
    for (int k = threadIdx.y; k < 64; k += blockDim.y) {
        const int r = r0 + k, c = c0 + 2 * tx;
        bf16 v0 = __float2bfloat16_rn(0.f), v1 = v0;
        if (r < rows) {
            if (pair_in && c + 1 < cols) {
                const __nv_bfloat162 q = *reinterpret_cast<const __nv_bfloat162*>(in + (size_t)r * cols + c);
                v0 = q.x;
                v1 = q.y;
            } else {
                if (c < cols) v0 = in[(size_t)r * cols + c];
                if (c + 1 < cols) v1 = in[(size_t)r * cols + c + 1];
            }
        }
        tile[k][2 * tx] = v0;
        tile[k][2 * tx + 1] = v1;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 64; k += blockDim.y) {
        const int c = c0 + k, r = r0 + 2 * tx;
        if (c >= cols) continue;
        const bf16 v0 = tile[2 * tx][k], v1 = tile[2 * tx + 1][k];
        if (pair_out && r + 1 < rows) {
            __nv_bfloat162 q;
            q.x = v0;
            q.y = v1;
            *reinterpret_cast<__nv_bfloat162*>(out + (size_t)c * rows + r) = q;
        } else {
            if (r < rows) out[(size_t)c * rows + r] = v0;
            if (r + 1 < rows) out[(size_t)c * rows + r + 1] = v1;
        }
    }
}

// 32 x 32 tiles of single BF16 elements: more blocks, for small matrices
__global__ void k_transpose32(const bf16* __restrict__ in, bf16* __restrict__ out, int rows, int cols) {
    __shared__ bf16 tile[32][34];
    const int c = blockIdx.x * 32 + threadIdx.x;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = blockIdx.y * 32 + k;
        if (r < rows && c < cols) tile[k][threadIdx.x] = in[(size_t)r * cols + c];
    }
    __syncthreads();
    const int r2 = blockIdx.y * 32 + threadIdx.x;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int c2 = blockIdx.x * 32 + k;
        if (c2 < cols && r2 < rows) out[(size_t)c2 * rows + r2] = tile[threadIdx.x][k];
    }
}

void transpose(const bf16* in, bf16* out, int rows, int cols, cudaStream_t st) {
    if ((long long)rows * cols < (1LL << 22)) {
        k_transpose32<<<dim3((cols + 31) / 32, (rows + 31) / 32), dim3(32, 8), 0, st>>>(in, out, rows, cols);
        return;
    }
    dim3 grid((cols + 63) / 64, (rows + 63) / 64), block(32, 8);
    k_transpose<<<grid, block, 0, st>>>(in, out, rows, cols);
}

__global__ void k_to_bf16(const float* __restrict__ in, bf16* __restrict__ out, long long count) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count; t += (long long)gridDim.x * blockDim.x)
        out[t] = __float2bfloat16_rn(in[t]);
}

// Loss gradient of the mean squared error against standardised targets:
// dY = 2 (Y - (T - mean)/std) / (B * D); per-block partial sums of the squared error.
// Y and dY have rows of Dp >= D entries (the extra ones get dY = 0); T has rows of D.
// Block (bx, row) takes columns bx*256 + threadIdx.x, stepping by gridDim.x*256.
__global__ void k_mse(const float* __restrict__ Y, const float* __restrict__ T, const float* __restrict__ mean,
                      const float* __restrict__ stdv, int B, int D, int Dp, bf16* __restrict__ dY,
                      double* __restrict__ part) {
    __shared__ double sh[8];
    const int row = blockIdx.y;
    const float scale = 2.0f / ((float)B * (float)D);
    const float* y = Y + (size_t)row * Dp;
    const float* t = T + (size_t)row * D;
    bf16* dy = dY + (size_t)row * Dp;
    double acc = 0.0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < Dp; j += gridDim.x * blockDim.x) {
        float r = 0.f;
        if (j < D) r = y[j] - (t[j] - mean[j]) / stdv[j];
        acc += (double)r * (double)r;
        dy[j] = __float2bfloat16_rn(scale * r);
    }
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
        part[(size_t)row * gridDim.x + blockIdx.x] = s;
    }
}

// out = scale * sum of n partial sums, one block of 256 threads, fixed order.
__global__ void k_sum_parts(const double* __restrict__ part, int n, double scale, double* __restrict__ out) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0] * scale;
}

// dZ = dH * (H > 0) (ReLU backward), FP32 in, BF16 out.
__global__ void k_relu_bwd(const float* __restrict__ dH, const bf16* __restrict__ H, bf16* __restrict__ dZ, long long count) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count; t += (long long)gridDim.x * blockDim.x)
        dZ[t] = __float2bfloat16_rn(__bfloat162float(H[t]) > 0.f ? dH[t] : 0.f);
}

// db[j] = sum over rows of G[row][j] (fixed order): block of 32 columns x 8 warps, warp w sums
// rows w, w+8, ...; the eight partial sums are added in warp order.
__global__ void k_colsum(const bf16* __restrict__ G, int rows, int cols, float* __restrict__ db) {
    __shared__ float sh[8][32];
    const int j = blockIdx.x * 32 + threadIdx.x, w = threadIdx.y;
    float s = 0.f;
    if (j < cols)
        for (int r = w; r < rows; r += 8) s += __bfloat162float(G[(size_t)r * cols + j]);
    sh[w][threadIdx.x] = s;
    __syncthreads();
    if (w == 0 && j < cols) {
        float t = 0.f;
        for (int q = 0; q < 8; ++q) t += sh[q][threadIdx.x];
        db[j] = t;
    }
}

// Adam (Kingma & Ba) on FP32 master weights; refreshes the BF16 copy.
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       bf16* __restrict__ wh, long long count, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count; t += (long long)gridDim.x * blockDim.x) {
        const float gt = g[t];
        const float mt = b1 * m[t] + (1.f - b1) * gt;
        const float vt = b2 * v[t] + (1.f - b2) * gt * gt;
        m[t] = mt;
        v[t] = vt;
        const float wn = w[t] - lr * (mt / c1) / (sqrtf(vt / c2) + eps);
        w[t] = wn;
        if (wh) wh[t] = __float2bfloat16_rn(wn);
    }
}

// Y * std + mean (undo the target standardisation), FP32; block (bx, row) as in k_mse.
__global__ void k_denorm(float* __restrict__ Y, const float* __restrict__ mean, const float* __restrict__ stdv, int B,
                         int D) {
    float* y = Y + (size_t)blockIdx.y * D;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < D; j += gridDim.x * blockDim.x) y[j] = y[j] * stdv[j] + mean[j];
}

// Per-output mean and standard deviation of a target matrix T [count][D] (row-major FP32): block
// (bx, p) takes 256 columns and the p-th slice of the rows, sums t - T[0][j] (a shift that keeps the
// sums small) and its square in FP32 over runs of 32 rows and adds each run into FP64.
__global__ void k_colstats_part(const float* __restrict__ T, long long count, int D, long long rows_per_part,
                                double* __restrict__ part) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= D) return;
    const long long r0 = blockIdx.y * rows_per_part;
    const long long r1 = min(count, r0 + rows_per_part);
    const float shift = T[j];
    double s1 = 0.0, s2 = 0.0;
    for (long long r = r0; r < r1; r += 32) {
        const long long re = min(r1, r + 32);
        float a1 = 0.f, a2 = 0.f;
        for (long long q = r; q < re; ++q) {
            const float d = T[q * D + j] - shift;
            a1 += d;
            a2 = fmaf(d, d, a2);
        }
        s1 += a1;
        s2 += a2;
    }
    part[((long long)blockIdx.y * D + j) * 2] = s1;
    part[((long long)blockIdx.y * D + j) * 2 + 1] = s2;
}

// mean_j = shift + S1/count, std_j = max(sqrt(S2/count - (S1/count)^2), min_std).
__global__ void k_colstats_final(const float* __restrict__ T, const double* __restrict__ part, int parts,
                                 long long count, int D, float min_std, float* __restrict__ mean,
                                 float* __restrict__ stdv) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= D) return;
    double s1 = 0.0, s2 = 0.0;
    for (int p = 0; p < parts; ++p) {
        s1 += part[((long long)p * D + j) * 2];
        s2 += part[((long long)p * D + j) * 2 + 1];
    }
    const double m1 = s1 / (double)count;
    const double var = fmax(s2 / (double)count - m1 * m1, 0.0);
    mean[j] = (float)((double)T[j] + m1);
    stdv[j] = fmaxf((float)sqrt(var), min_std);
}

// blocks per row for the row-wise kernels (grid y = rows): about 1184 blocks in all
inline int row_blocks(int cols, int rows) {
    return std::max(1, std::min((cols + 255) / 256, 148 * 8 / std::max(rows, 1)));
}

inline int grid1(long long count) {
    return (int)std::max<long long>(1, std::min<long long>((count + 255) / 256, 148 * 8));
}

}  // namespace

struct mfs_mlp {
    int din = 0, width = 0, dout = 0, maxb = 0;
    int doutp = 0;  // dout rounded up to a multiple of 8 (16-byte rows); the extra outputs stay zero
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    int step = 0;
    float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
    // parameters: FP32 master, Adam moments, BF16 copies; index 0..2 = layers 1..3
    float *W[3] = {}, *b[3] = {}, *mW[3] = {}, *vW[3] = {}, *mb[3] = {}, *vb[3] = {};
    bf16 *Wh[3] = {}, *Wt[3] = {};
    float *gW[3] = {}, *gb[3] = {};
    float *mean = nullptr, *stdv = nullptr;
    // activations and gradients
    bf16 *X = nullptr, *H1 = nullptr, *H2 = nullptr, *dY = nullptr, *dYt = nullptr, *H2t = nullptr, *H1t = nullptr,
         *Xt = nullptr, *dZ2 = nullptr, *dZ2t = nullptr, *dZ1 = nullptr, *dZ1t = nullptr;
    float *Y = nullptr, *dH = nullptr, *work = nullptr;
    bool wt2_fresh = false;  // Wt[2] holds the transpose of the current Wh[2]
    bool keep_grads = false; // mfs_mlp_train_step also stores layer 3's weight gradient
    double *loss_part = nullptr, *loss = nullptr;
    int* err = nullptr;
    size_t work_floats = 0;
    std::vector<void*> allocs;
    std::string last_error;
};

namespace {

thread_local std::string g_mlp_error;

mfs_status mfail(mfs_mlp* s, mfs_status st, const std::string& msg) {
    if (s)
        s->last_error = msg;
    else
        g_mlp_error = msg;
    return st;
}

template <typename T>
mfs_status malloc_zero(mfs_mlp* s, T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = mfs::device_malloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return mfail(s, MFS_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    s->allocs.push_back(q);
    *p = static_cast<T*>(q);
    e = cudaMemsetAsync(q, 0, std::max<size_t>(count, 1) * sizeof(T), s->stream);
    if (e != cudaSuccess) return mfail(s, MFS_ERR_CUDA, std::string("cudaMemset: ") + cudaGetErrorString(e));
    return MFS_OK;
}

#define MTRY(x)                         \
    do {                                \
        mfs_status st_ = (x);           \
        if (st_ != MFS_OK) return st_;  \
    } while (0)

int layer_in(const mfs_mlp* s, int l) { return l == 0 ? s->din : s->width; }
int layer_out(const mfs_mlp* s, int l) { return l == 2 ? s->doutp : s->width; }
int user_out(const mfs_mlp* s, int l) { return l == 2 ? s->dout : s->width; }

mfs_status check_err(mfs_mlp* s) {
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, s->err, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return mfail(s, MFS_ERR_CUDA, std::string("mlp: ") + cudaGetErrorString(e));
    if (h) {
        cudaMemsetAsync(s->err, 0, sizeof(int), s->stream);
        return mfail(s, MFS_ERR_TIMEOUT, "mlp: a bounded wait in the tensor-core GEMM gave up");
    }
    return MFS_OK;
}

mfs_status run_gemm(mfs_mlp* s, int M, int N, int K, const bf16* A, const bf16* B, const float* bias, int relu,
                    int out_fp32, void* C, int splits) {
    std::string why;
    mfs_status st = gemm(M, N, K, A, B, bias, relu, out_fp32, C, splits, s->work, s->err, s->stream, &why);
    if (st != MFS_OK) return mfail(s, st, why);
    return MFS_OK;
}

int splits_for(const mfs_mlp* s, int M, int N, int K) {
    // enough CTAs to cover the GPU when M x N is small and K long; bounded by the workspace
    const int tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
    int sp = std::max(1, std::min((K + BK - 1) / BK, 2 * 148 / std::max(1, tiles)));
    while (sp > 1 && (size_t)sp * M * N > s->work_floats) --sp;
    return sp;
}

// forward for a batch already converted to BF16 in s->X; output (standardised) in s->Y
mfs_status forward_bf16(mfs_mlp* s, int B) {
    MTRY(run_gemm(s, B, s->width, s->din, s->X, s->Wh[0], s->b[0], 1, 0, s->H1, 1));
    MTRY(run_gemm(s, B, s->width, s->width, s->H1, s->Wh[1], s->b[1], 1, 0, s->H2,
                  splits_for(s, B, s->width, s->width)));
    MTRY(run_gemm(s, B, s->doutp, s->width, s->H2, s->Wh[2], s->b[2], 0, 1, s->Y, 1));
    return MFS_OK;
}

}  // namespace

extern "C" {

mfs_status mfs_mlp_create(int32_t din, int32_t width, int32_t dout, int32_t max_batch, uint64_t seed, void* cuda_stream,
                          mfs_mlp** out) {
    g_mlp_error.clear();
    if (!out) return mfail(nullptr, MFS_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (din < 1 || width < 1 || dout < 1 || max_batch < 1 || din % 8 || width % 8 || max_batch % 8 ||
        max_batch > 65535)
        return mfail(nullptr, MFS_ERR_INVALID,
                     "din, width and max_batch must be positive multiples of 8 (max_batch <= 65535), dout >= 1");
    mfs_mlp* s = new (std::nothrow) mfs_mlp();
    if (!s) return mfail(nullptr, MFS_ERR_OOM, "host allocation failed");
    auto bail = [&](mfs_status st) {
        g_mlp_error = s->last_error;
        mfs_mlp_destroy(s);
        return st;
    };
    s->din = din;
    s->width = width;
    s->dout = dout;
    s->doutp = (dout + 7) / 8 * 8;
    s->maxb = max_batch;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) {
        if (cuda_stream)
            s->stream = static_cast<cudaStream_t>(cuda_stream);
        else {
            e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
            s->own_stream = true;
        }
    }
    if (e != cudaSuccess) {
        s->last_error = std::string("CUDA set-up: ") + cudaGetErrorString(e);
        return bail(MFS_ERR_CUDA);
    }
    if (!encode_fn()) {
        s->last_error = "cuTensorMapEncodeTiled is not available from the driver";
        return bail(MFS_ERR_CUDA);
    }
#define MCHK(x)                             \
    do {                                    \
        mfs_status q_ = (x);                \
        if (q_ != MFS_OK) return bail(q_);  \
    } while (0)
    // He-uniform initial weights from a fixed LCG-free generator (splitmix64), zero biases
    uint64_t state = seed ^ 0x9E3779B97F4A7C15ull;
    auto next = [&]() {
        uint64_t z = (state += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    for (int l = 0; l < 3; ++l) {
        const int fi = layer_in(s, l), fo = layer_out(s, l);
        const size_t cnt = (size_t)fi * fo;
        MCHK(malloc_zero(s, &s->W[l], cnt));
        MCHK(malloc_zero(s, &s->mW[l], cnt));
        MCHK(malloc_zero(s, &s->vW[l], cnt));
        MCHK(malloc_zero(s, &s->gW[l], cnt));
        MCHK(malloc_zero(s, &s->Wh[l], cnt));
        MCHK(malloc_zero(s, &s->Wt[l], cnt));
        MCHK(malloc_zero(s, &s->b[l], fo));
        MCHK(malloc_zero(s, &s->mb[l], fo));
        MCHK(malloc_zero(s, &s->vb[l], fo));
        MCHK(malloc_zero(s, &s->gb[l], fo));
        std::vector<float> h(cnt, 0.0f);
        const double lim = std::sqrt(6.0 / fi) * (l == 2 ? 0.1 : 1.0);
        const size_t live = (size_t)fi * user_out(s, l);
        for (size_t i = 0; i < live; ++i) h[i] = (float)((2.0 * ((next() >> 11) * (1.0 / 9007199254740992.0)) - 1.0) * lim);
        e = cudaMemcpyAsync(s->W[l], h.data(), cnt * sizeof(float), cudaMemcpyHostToDevice, s->stream);
        if (e != cudaSuccess) {
            s->last_error = "upload";
            return bail(MFS_ERR_CUDA);
        }
        k_to_bf16<<<grid1(cnt), 256, 0, s->stream>>>(s->W[l], s->Wh[l], (long long)cnt);
    }
    const int B = max_batch;
    const int Dp = s->doutp;
    MCHK(malloc_zero(s, &s->mean, Dp));
    MCHK(malloc_zero(s, &s->stdv, Dp));
    {
        std::vector<float> ones(Dp, 1.0f);
        cudaMemcpyAsync(s->stdv, ones.data(), Dp * sizeof(float), cudaMemcpyHostToDevice, s->stream);
    }
    MCHK(malloc_zero(s, &s->X, (size_t)B * din));
    MCHK(malloc_zero(s, &s->Xt, (size_t)B * din));
    MCHK(malloc_zero(s, &s->H1, (size_t)B * width));
    MCHK(malloc_zero(s, &s->H2, (size_t)B * width));
    MCHK(malloc_zero(s, &s->H1t, (size_t)B * width));
    MCHK(malloc_zero(s, &s->H2t, (size_t)B * width));
    MCHK(malloc_zero(s, &s->Y, (size_t)B * Dp));
    MCHK(malloc_zero(s, &s->dY, (size_t)B * Dp));
    MCHK(malloc_zero(s, &s->dYt, (size_t)B * Dp));
    MCHK(malloc_zero(s, &s->dH, (size_t)B * width));
    MCHK(malloc_zero(s, &s->dZ2, (size_t)B * width));
    MCHK(malloc_zero(s, &s->dZ2t, (size_t)B * width));
    MCHK(malloc_zero(s, &s->dZ1, (size_t)B * width));
    MCHK(malloc_zero(s, &s->dZ1t, (size_t)B * width));
    s->work_floats = (size_t)64 * B * width;
    MCHK(malloc_zero(s, &s->work, s->work_floats));
    // partial loss sums: k_mse's blocks, or one per output tile of the fused loss epilogue
    const size_t tiles = (size_t)((Dp + BN - 1) / BN) * ((max_batch + BM - 1) / BM);
    MCHK(malloc_zero(s, &s->loss_part, std::max<size_t>(std::max(148 * 8, max_batch), tiles)));
    MCHK(malloc_zero(s, &s->loss, 1));
    MCHK(malloc_zero(s, &s->err, 1));
    e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        s->last_error = std::string("set-up: ") + cudaGetErrorString(e);
        return bail(MFS_ERR_CUDA);
    }
#undef MCHK
    *out = s;
    return MFS_OK;
}

void mfs_mlp_destroy(mfs_mlp* s) {
    if (!s) return;
    cudaSetDevice(s->device);
    if (s->stream) cudaStreamSynchronize(s->stream);
    for (void* p : s->allocs) cudaFree(p);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

const char* mfs_mlp_last_error(const mfs_mlp* s) {
    return s ? s->last_error.c_str() : g_mlp_error.c_str();
}

mfs_status mfs_mlp_set_output_scaling(mfs_mlp* s, const float* mean, const float* stdv) {
    if (!s || !mean || !stdv) return MFS_ERR_INVALID;
    for (int j = 0; j < s->dout; ++j)
        if (!(stdv[j] > 0.f) || !std::isfinite(stdv[j]) || !std::isfinite(mean[j]))
            return mfail(s, MFS_ERR_INVALID, "output scaling: std must be positive and finite");
    cudaError_t e = cudaMemcpyAsync(s->mean, mean, s->dout * sizeof(float), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->stdv, stdv, s->dout * sizeof(float), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return e == cudaSuccess ? MFS_OK : mfail(s, MFS_ERR_CUDA, cudaGetErrorString(e));
}

mfs_status mfs_mlp_fit_output_scaling(mfs_mlp* s, int64_t count, const float* targets, float min_std) {
    if (!s || !targets || count < 1 || !(min_std > 0.f) || !std::isfinite(min_std)) return MFS_ERR_INVALID;
    cudaSetDevice(s->device);
    const int D = s->dout;
    const int parts = (int)std::min<long long>(64, (count + 255) / 256);
    const long long per = (count + parts - 1) / parts;
    double* part = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&part), (size_t)parts * D * 2 * sizeof(double), s->stream);
    if (e != cudaSuccess) return mfail(s, MFS_ERR_OOM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
    k_colstats_part<<<dim3((D + 255) / 256, parts), 256, 0, s->stream>>>(targets, count, D, per, part);
    k_colstats_final<<<(D + 255) / 256, 256, 0, s->stream>>>(targets, part, parts, count, D, min_std, s->mean,
                                                             s->stdv);
    e = cudaGetLastError();
    cudaFreeAsync(part, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return e == cudaSuccess ? MFS_OK : mfail(s, MFS_ERR_CUDA, cudaGetErrorString(e));
}

mfs_status mfs_mlp_get_output_scaling(mfs_mlp* s, float* mean, float* stdv) {
    if (!s) return MFS_ERR_INVALID;
    cudaSetDevice(s->device);
    cudaError_t e = cudaSuccess;
    if (mean) e = cudaMemcpyAsync(mean, s->mean, s->dout * sizeof(float), cudaMemcpyDeviceToHost, s->stream);
    if (stdv && e == cudaSuccess)
        e = cudaMemcpyAsync(stdv, s->stdv, s->dout * sizeof(float), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return e == cudaSuccess ? MFS_OK : mfail(s, MFS_ERR_CUDA, cudaGetErrorString(e));
}

mfs_status mfs_mlp_forward(mfs_mlp* s, int32_t batch, const float* x, float* y, int32_t denormalize) {
    MFS_TRACE("mfs_mlp_forward");
    if (!s || !x || !y || batch < 1 || batch > s->maxb) return MFS_ERR_INVALID;
    cudaSetDevice(s->device);
    k_to_bf16<<<grid1((long long)batch * s->din), 256, 0, s->stream>>>(x, s->X, (long long)batch * s->din);
    MTRY(forward_bf16(s, batch));
    if (denormalize)
        k_denorm<<<dim3(row_blocks(s->doutp, batch), batch), 256, 0, s->stream>>>(s->Y, s->mean, s->stdv, batch,
                                                                                     s->doutp);
    if (cudaMemcpy2DAsync(y, (size_t)s->dout * sizeof(float), s->Y, (size_t)s->doutp * sizeof(float),
                          (size_t)s->dout * sizeof(float), batch, cudaMemcpyDeviceToDevice, s->stream) != cudaSuccess)
        return mfail(s, MFS_ERR_CUDA, "copy of the output");
    return check_err(s);
}

// Loss and gradients of one batch (no update); the gradients stay in the MLP (mfs_mlp_get_grads).
mfs_status mfs_mlp_backward(mfs_mlp* s, int32_t batch, const float* x, const float* target, double* loss) {
    MFS_TRACE("mfs_mlp_backward");
    if (!s || !x || !target || batch < 1 || batch > s->maxb || batch % 8) return MFS_ERR_INVALID;
    cudaSetDevice(s->device);
    const int B = batch, W = s->width, D = s->doutp, I = s->din;
    cudaStream_t st = s->stream;
    k_to_bf16<<<grid1((long long)B * I), 256, 0, st>>>(x, s->X, (long long)B * I);
    MTRY(forward_bf16(s, B));
    const int lb = row_blocks(D, B);  // blocks per row of k_mse; lb * B <= max(1184, B) partial sums
    k_mse<<<dim3(lb, B), 256, 0, st>>>(s->Y, target, s->mean, s->stdv, B, s->dout, D, s->dY, s->loss_part);
    k_sum_parts<<<1, 256, 0, st>>>(s->loss_part, lb * B, 1.0 / ((double)B * s->dout), s->loss);
    // layer 3: dW3 = dY^T H2, db3 = colsum(dY), dH2 = dY W3
    transpose(s->dY, s->dYt, B, D, st);
    transpose(s->H2, s->H2t, B, W, st);
    MTRY(run_gemm(s, D, W, B, s->dYt, s->H2t, nullptr, 0, 1, s->gW[2], 1));
    k_colsum<<<(D + 31) / 32, dim3(32, 8), 0, st>>>(s->dY, B, D, s->gb[2]);
    transpose(s->Wh[2], s->Wt[2], D, W, st);
    s->wt2_fresh = true;
    MTRY(run_gemm(s, B, W, D, s->dY, s->Wt[2], nullptr, 0, 1, s->dH, splits_for(s, B, W, D)));
    k_relu_bwd<<<grid1((long long)B * W), 256, 0, st>>>(s->dH, s->H2, s->dZ2, (long long)B * W);
    // layer 2
    transpose(s->dZ2, s->dZ2t, B, W, st);
    transpose(s->H1, s->H1t, B, W, st);
    MTRY(run_gemm(s, W, W, B, s->dZ2t, s->H1t, nullptr, 0, 1, s->gW[1], 1));
    k_colsum<<<(W + 31) / 32, dim3(32, 8), 0, st>>>(s->dZ2, B, W, s->gb[1]);
    transpose(s->Wh[1], s->Wt[1], W, W, st);
    MTRY(run_gemm(s, B, W, W, s->dZ2, s->Wt[1], nullptr, 0, 1, s->dH, splits_for(s, B, W, W)));
    k_relu_bwd<<<grid1((long long)B * W), 256, 0, st>>>(s->dH, s->H1, s->dZ1, (long long)B * W);
    // layer 1
    transpose(s->dZ1, s->dZ1t, B, W, st);
    transpose(s->X, s->Xt, B, I, st);
    MTRY(run_gemm(s, W, I, B, s->dZ1t, s->Xt, nullptr, 0, 1, s->gW[0], 1));
    k_colsum<<<(W + 31) / 32, dim3(32, 8), 0, st>>>(s->dZ1, B, W, s->gb[0]);
    if (cudaGetLastError() != cudaSuccess) return mfail(s, MFS_ERR_CUDA, "mlp backward launch");
    if (loss && cudaMemcpyAsync(loss, s->loss, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return mfail(s, MFS_ERR_CUDA, "loss copy");
    return check_err(s);
}

// One Adam step with the gradients of the last mfs_mlp_backward.
mfs_status mfs_mlp_adam_step(mfs_mlp* s, float lr) {
    if (!s || !(lr > 0.f)) return MFS_ERR_INVALID;
    cudaSetDevice(s->device);
    ++s->step;
    const float c1 = 1.f - std::pow(s->beta1, (float)s->step), c2 = 1.f - std::pow(s->beta2, (float)s->step);
    for (int l = 0; l < 3; ++l) {
        const long long cw = (long long)layer_in(s, l) * layer_out(s, l), cb = layer_out(s, l);
        k_adam<<<grid1(cw), 256, 0, s->stream>>>(s->W[l], s->gW[l], s->mW[l], s->vW[l], s->Wh[l], cw, lr, s->beta1,
                                                 s->beta2, s->eps, c1, c2);
        k_adam<<<grid1(cb), 256, 0, s->stream>>>(s->b[l], s->gb[l], s->mb[l], s->vb[l], nullptr, cb, lr, s->beta1,
                                                 s->beta2, s->eps, c1, c2);
    }
    s->wt2_fresh = false;
    if (cudaGetLastError() != cudaSuccess) return mfail(s, MFS_ERR_CUDA, "adam launch");
    return check_err(s);
}

// One training step with the output layer fused into two GEMM epilogues: the forward GEMM of layer 3
// writes the loss gradient dY (and its transpose) instead of Y, and the weight-gradient GEMM of
// layer 3 applies Adam to W3 directly (its gradient is never stored). The other steps are those of
// mfs_mlp_backward followed by mfs_mlp_adam_step, in an order where dH2 still sees the old W3.
mfs_status mfs_mlp_train_step(mfs_mlp* s, int32_t batch, const float* x, const float* target, float lr, double* loss) {
    MFS_TRACE("mfs_mlp_train_step");
    if (!s || !x || !target || batch < 1 || batch > s->maxb || batch % 8 || !(lr > 0.f)) return MFS_ERR_INVALID;
    cudaSetDevice(s->device);
    const int B = batch, W = s->width, D = s->doutp, I = s->din;
    cudaStream_t st = s->stream;
    ++s->step;
    const float c1 = 1.f - std::pow(s->beta1, (float)s->step), c2 = 1.f - std::pow(s->beta2, (float)s->step);
    if (!s->wt2_fresh) {
        transpose(s->Wh[2], s->Wt[2], D, W, st);
        s->wt2_fresh = true;
    }
    k_to_bf16<<<grid1((long long)B * I), 256, 0, st>>>(x, s->X, (long long)B * I);
    MTRY(run_gemm(s, B, W, I, s->X, s->Wh[0], s->b[0], 1, 0, s->H1, 1));
    MTRY(run_gemm(s, B, W, W, s->H1, s->Wh[1], s->b[1], 1, 0, s->H2, splits_for(s, B, W, W)));
    // layer 3 forward + loss: dY, dY^T and the partial sums of the squared residuals
    GemmArgs fl{};
    fl.T = target;
    fl.ldT = s->dout;
    fl.dout = s->dout;
    fl.mean = s->mean;
    fl.stdv = s->stdv;
    fl.scale = 2.0f / ((float)B * (float)s->dout);
    fl.dYt = s->dYt;
    fl.ldt = B;
    fl.part = s->loss_part;
    {
        std::string why;
        mfs_status q = gemm(B, D, W, s->H2, s->Wh[2], s->b[2], 0, 0, s->dY, 1, s->work, s->err, st, &why, SPIN, 0,
                            EPI_LOSS, &fl);
        if (q != MFS_OK) return mfail(s, q, why);
    }
    const int tiles = ((D + BN - 1) / BN) * ((B + BM - 1) / BM);
    k_sum_parts<<<1, 256, 0, st>>>(s->loss_part, tiles, 1.0 / ((double)B * s->dout), s->loss);
    k_colsum<<<(D + 31) / 32, dim3(32, 8), 0, st>>>(s->dY, B, D, s->gb[2]);
    // dH2 = dY W3 (old W3), then layers 2 and 1 as in mfs_mlp_backward
    MTRY(run_gemm(s, B, W, D, s->dY, s->Wt[2], nullptr, 0, 1, s->dH, splits_for(s, B, W, D)));
    k_relu_bwd<<<grid1((long long)B * W), 256, 0, st>>>(s->dH, s->H2, s->dZ2, (long long)B * W);
    transpose(s->dZ2, s->dZ2t, B, W, st);
    transpose(s->H1, s->H1t, B, W, st);
    MTRY(run_gemm(s, W, W, B, s->dZ2t, s->H1t, nullptr, 0, 1, s->gW[1], 1));
    k_colsum<<<(W + 31) / 32, dim3(32, 8), 0, st>>>(s->dZ2, B, W, s->gb[1]);
    transpose(s->Wh[1], s->Wt[1], W, W, st);
    MTRY(run_gemm(s, B, W, W, s->dZ2, s->Wt[1], nullptr, 0, 1, s->dH, splits_for(s, B, W, W)));
    k_relu_bwd<<<grid1((long long)B * W), 256, 0, st>>>(s->dH, s->H1, s->dZ1, (long long)B * W);
    transpose(s->dZ1, s->dZ1t, B, W, st);
    transpose(s->X, s->Xt, B, I, st);
    MTRY(run_gemm(s, W, I, B, s->dZ1t, s->Xt, nullptr, 0, 1, s->gW[0], 1));
    k_colsum<<<(W + 31) / 32, dim3(32, 8), 0, st>>>(s->dZ1, B, W, s->gb[0]);
    // layer 3 weight gradient dY^T H2 with Adam in the epilogue (W3, moments, Wh3, Wt3)
    transpose(s->H2, s->H2t, B, W, st);
    GemmArgs fa{};
    fa.W = s->W[2];
    fa.mom = s->mW[2];
    fa.vel = s->vW[2];
    fa.Wh = s->Wh[2];
    fa.Wt = s->Wt[2];
    fa.ldt = D;
    fa.lr = lr;
    fa.b1 = s->beta1;
    fa.b2 = s->beta2;
    fa.eps = s->eps;
    fa.c1 = c1;
    fa.c2 = c2;
    fa.gkeep = s->keep_grads ? s->gW[2] : nullptr;
    {
        std::string why;
        mfs_status q = gemm(D, W, B, s->dYt, s->H2t, nullptr, 0, 1, nullptr, 1, s->work, s->err, st, &why, SPIN, 0,
                            EPI_ADAM, &fa);
        if (q != MFS_OK) return mfail(s, q, why);
    }
    // Adam on layers 1 and 2 and on all biases
    for (int l = 0; l < 3; ++l) {
        const long long cw = (long long)layer_in(s, l) * layer_out(s, l), cb = layer_out(s, l);
        if (l < 2)
            k_adam<<<grid1(cw), 256, 0, st>>>(s->W[l], s->gW[l], s->mW[l], s->vW[l], s->Wh[l], cw, lr, s->beta1,
                                              s->beta2, s->eps, c1, c2);
        k_adam<<<grid1(cb), 256, 0, st>>>(s->b[l], s->gb[l], s->mb[l], s->vb[l], nullptr, cb, lr, s->beta1, s->beta2,
                                          s->eps, c1, c2);
    }
    if (cudaGetLastError() != cudaSuccess) return mfail(s, MFS_ERR_CUDA, "mlp train step launch");
    if (loss && cudaMemcpyAsync(loss, s->loss, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return mfail(s, MFS_ERR_CUDA, "loss copy");
    return check_err(s);
}

// Host copies of layer l's FP32 master weights [out][in] and bias (either may be NULL); set copies
// them in and refreshes the BF16 copy. Gradients of the last backward pass likewise.
mfs_status mfs_mlp_get_params(mfs_mlp* s, int32_t l, float* W, float* b) {
    if (!s || l < 0 || l > 2) return MFS_ERR_INVALID;
    const size_t cw = (size_t)layer_in(s, l) * user_out(s, l), cb = user_out(s, l);
    if (W && cudaMemcpy(W, s->W[l], cw * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return MFS_ERR_CUDA;
    if (b && cudaMemcpy(b, s->b[l], cb * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return MFS_ERR_CUDA;
    return MFS_OK;
}

mfs_status mfs_mlp_set_params(mfs_mlp* s, int32_t l, const float* W, const float* b) {
    if (!s || l < 0 || l > 2) return MFS_ERR_INVALID;
    const size_t cw = (size_t)layer_in(s, l) * user_out(s, l), cb = user_out(s, l);
    if (W) {
        if (cudaMemcpy(s->W[l], W, cw * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return MFS_ERR_CUDA;
        k_to_bf16<<<grid1(cw), 256, 0, s->stream>>>(s->W[l], s->Wh[l], (long long)cw);
        if (l == 2) s->wt2_fresh = false;
    }
    if (b && cudaMemcpy(s->b[l], b, cb * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return MFS_ERR_CUDA;
    return cudaStreamSynchronize(s->stream) == cudaSuccess ? MFS_OK : MFS_ERR_CUDA;
}

mfs_status mfs_mlp_get_grads(mfs_mlp* s, int32_t l, float* gW, float* gb) {
    if (!s || l < 0 || l > 2) return MFS_ERR_INVALID;
    const size_t cw = (size_t)layer_in(s, l) * user_out(s, l), cb = user_out(s, l);
    if (gW && cudaMemcpy(gW, s->gW[l], cw * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return MFS_ERR_CUDA;
    if (gb && cudaMemcpy(gb, s->gb[l], cb * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return MFS_ERR_CUDA;
    return MFS_OK;
}

mfs_status mfs_mlp_keep_grads(mfs_mlp* s, int32_t on) {
    if (!s) return MFS_ERR_INVALID;
    s->keep_grads = on != 0;
    return MFS_OK;
}

// Adam state of layer l: first and second moments of the weights [out][in] and of the bias (any
// may be NULL) and the number of steps taken.
mfs_status mfs_mlp_get_adam_state(mfs_mlp* s, int32_t l, float* mW, float* vW, float* mb, float* vb, int64_t* step) {
    if (!s || l < 0 || l > 2) return MFS_ERR_INVALID;
    const size_t cw = (size_t)layer_in(s, l) * user_out(s, l), cb = user_out(s, l);
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return MFS_ERR_CUDA;
    if (mW && cudaMemcpy(mW, s->mW[l], cw * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return MFS_ERR_CUDA;
    if (vW && cudaMemcpy(vW, s->vW[l], cw * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return MFS_ERR_CUDA;
    if (mb && cudaMemcpy(mb, s->mb[l], cb * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return MFS_ERR_CUDA;
    if (vb && cudaMemcpy(vb, s->vb[l], cb * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) return MFS_ERR_CUDA;
    if (step) *step = s->step;
    return MFS_OK;
}

// The BF16 copy of layer l's weights [out][in] that the GEMMs read, as raw 16-bit patterns.
mfs_status mfs_mlp_get_weights_bf16(mfs_mlp* s, int32_t l, uint16_t* Wh) {
    if (!s || l < 0 || l > 2 || !Wh) return MFS_ERR_INVALID;
    const size_t cw = (size_t)layer_in(s, l) * user_out(s, l);
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return MFS_ERR_CUDA;
    if (cudaMemcpy(Wh, s->Wh[l], cw * sizeof(uint16_t), cudaMemcpyDeviceToHost) != cudaSuccess) return MFS_ERR_CUDA;
    return MFS_OK;
}

// Stand-alone tensor-core GEMM through the C ABI (device pointers): C = A B^T (+ bias, ReLU).
mfs_status mfs_gemm_bf16_wait_test(void* cuda_stream) {
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int M = 128, N = 128, K = 64;
    void *A = nullptr, *B = nullptr, *C = nullptr;
    int* err = nullptr;
    mfs_status out = MFS_ERR_CUDA;
    if (cudaMalloc(&A, M * K * 2) == cudaSuccess && cudaMalloc(&B, N * K * 2) == cudaSuccess &&
        cudaMalloc(&C, M * N * 4) == cudaSuccess && cudaMalloc(reinterpret_cast<void**>(&err), sizeof(int)) == cudaSuccess &&
        cudaMemsetAsync(A, 0, M * K * 2, st) == cudaSuccess && cudaMemsetAsync(B, 0, N * K * 2, st) == cudaSuccess &&
        cudaMemsetAsync(err, 0, sizeof(int), st) == cudaSuccess) {
        std::string why;
        // the one-tile kernel, then the persistent one (the loss epilogue) with no loads issued:
        // both must report the timeout
        auto result = [&](mfs_status launched) -> mfs_status {
            int h = 0;
            if (launched != MFS_OK) return launched;
            if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
                return MFS_ERR_CUDA;
            return h == ERR_TIMEOUT ? MFS_ERR_TIMEOUT : (h ? MFS_ERR_CUDA : MFS_OK);
        };
        out = result(gemm(M, N, K, static_cast<bf16*>(A), static_cast<bf16*>(B), nullptr, 0, 1, C, 1, nullptr, err, st,
                          &why, 1024u, 1));
        float *T = nullptr, *mv = nullptr;
        void* dYt = nullptr;
        double* part = nullptr;
        if (out == MFS_ERR_TIMEOUT) {
            out = MFS_ERR_CUDA;
            if (cudaMalloc(reinterpret_cast<void**>(&T), M * N * 4) == cudaSuccess &&
                cudaMalloc(reinterpret_cast<void**>(&mv), 2 * N * 4) == cudaSuccess &&
                cudaMalloc(&dYt, M * N * 2) == cudaSuccess &&
                cudaMalloc(reinterpret_cast<void**>(&part), 64 * sizeof(double)) == cudaSuccess &&
                cudaMemsetAsync(T, 0, M * N * 4, st) == cudaSuccess && cudaMemsetAsync(mv, 0, 2 * N * 4, st) == cudaSuccess) {
                GemmArgs fa{};
                fa.T = T;
                fa.ldT = N;
                fa.dout = N;
                fa.mean = mv;
                fa.stdv = mv + N;
                fa.scale = 1.f;
                fa.dYt = static_cast<bf16*>(dYt);
                fa.ldt = M;
                fa.part = part;
                out = result(gemm(M, N, K, static_cast<bf16*>(A), static_cast<bf16*>(B), nullptr, 0, 0, C, 1, nullptr, err,
                                  st, &why, 1024u, 1, EPI_LOSS, &fa));
            }
        }
        cudaStreamSynchronize(st);
        cudaFree(T);
        cudaFree(mv);
        cudaFree(dYt);
        cudaFree(part);
    }
    cudaStreamSynchronize(st);
    cudaFree(A);
    cudaFree(B);
    cudaFree(C);
    cudaFree(err);
    return out;
}

mfs_status mfs_gemm_bf16(int64_t M, int64_t N, int64_t K, const void* A, const void* B, const float* bias, int32_t relu,
                         int32_t out_fp32, void* C, int32_t splits, void* cuda_stream) {
    if (M < 0 || N < 0 || K < 0 || M >= INT32_MAX || N >= INT32_MAX || K >= INT32_MAX || !A || !B || !C)
        return MFS_ERR_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int* err = nullptr;
    float* work = nullptr;
    if (cudaMallocAsync((void**)&err, sizeof(int), st) != cudaSuccess) return MFS_ERR_OOM;
    cudaMemsetAsync(err, 0, sizeof(int), st);
    splits = std::max(1, (int)splits);
    if (splits > 1 && cudaMallocAsync((void**)&work, (size_t)splits * M * N * sizeof(float), st) != cudaSuccess) {
        cudaFreeAsync(err, st);
        return MFS_ERR_OOM;
    }
    std::string why;
    mfs_status s = gemm((int)M, (int)N, (int)K, static_cast<const bf16*>(A), static_cast<const bf16*>(B), bias, relu,
                        out_fp32, C, splits, work, err, st, &why);
    int h = 0;
    cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (work) cudaFreeAsync(work, st);
    cudaFreeAsync(err, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return MFS_ERR_CUDA;
    if (s != MFS_OK) return s;
    return h ? MFS_ERR_TIMEOUT : MFS_OK;
}

}  // extern "C"
